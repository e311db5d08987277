// bin_rays_static: the binning entry point for callers that cannot allocate
// device memory.
//
// Some hosts own every byte of device memory through their own pool (an
// engine with a fixed, pre-reserved budget) or have no device allocator at all
// to carve a workspace from (a plain C caller of this ABI).  They cannot call
// cudaMalloc, nor hand bin_rays the workspace it asks for.  This variant runs
// the same binning kernels with its scratch in a file-scope device array of
// fixed size, reserved when this library's module is loaded on a device and
// held by that device until the process exits.  It calls no cudaMalloc,
// cudaFree or allocating routine.
#include <mutex>
#include <string>

#include "common.cuh"
#include "svo.cuh"

namespace wfpg {
size_t bin_workspace_bytes(const wfpg_svo* s, uint32_t n, int mode, uint32_t n_sizes);
int bin_rays_impl(const wfpg_svo* s, const float* pos, const float* nrm, uint32_t n, const wfpg_bin_params* p,
                  const uint32_t* sizes, uint32_t* bin_of_ray, uint32_t* ray_order, uint32_t* bin_offset,
                  uint32_t* origin_ray, uint32_t bin_cap, uint32_t* n_bins_dev, void* workspace, size_t ws_bytes,
                  cudaStream_t st, const uint32_t* frame_dev = nullptr);
int set_last_error(int code, const std::string& msg);
}  // namespace wfpg

// the shared scratch: one copy per device that loads this library
static __device__ __align__(256) unsigned char g_bin_static_scratch[WFPG_BIN_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

int static_fail(int code, const std::string& msg) { return wfpg::set_last_error(code, msg); }

// Device address of the scratch array on the current device.  The first call
// per device looks it up (the host-side name of the array is only a stand-in
// for the device copy); later calls reuse the cached address.
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return static_fail(WFPG_ERR_CUDA, "bin_rays_static: no usable current device");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_static_scratch);
        if (e != cudaSuccess || !p)
            return static_fail(WFPG_ERR_CUDA, std::string("bin_rays_static: cudaGetSymbolAddress failed: ") +
                                                  cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return WFPG_OK;
}
}  // namespace

extern "C" {

int bin_rays_static(const wfpg_svo* s, const float* pos, const float* nrm, uint32_t n, const wfpg_bin_params* p,
                    const uint32_t* sizes, uint32_t* bin_of_ray, uint32_t* ray_order, uint32_t* bin_offset,
                    uint32_t* origin_ray, uint32_t bin_cap, uint32_t* n_bins_dev, void* stream) {
    if (!s || !p) return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: null svo or params");
    if (p->mode != WFPG_BIN_PARTITION_S && p->mode != WFPG_BIN_RUNS)
        return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: unknown mode");
    if (n >= 0x80000000u) return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: at most 2^31 - 1 rays");
    if (n && (!pos || !bin_of_ray || !ray_order))
        return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: null ray array");
    if (!bin_offset || !n_bins_dev || (bin_cap && !origin_ray))
        return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: null bin array");
    if (p->mode == WFPG_BIN_RUNS) {
        if (n && !nrm) return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: RUNS mode needs nrm");
        if (p->n_sizes == 0 || !sizes) return static_fail(WFPG_ERR_INVALID_ARG, "bin_rays_static: RUNS mode needs sizes");
        if (p->n_sizes > bin_cap) return static_fail(WFPG_ERR_CAPACITY, "bin_rays_static: n_sizes exceeds bin_cap");
    }
    const size_t need = wfpg::bin_workspace_bytes(s, n, p->mode, p->n_sizes);
    if (need > (size_t)WFPG_BIN_STATIC_SCRATCH_BYTES)
        return static_fail(WFPG_ERR_CAPACITY,
                           "bin_rays_static: this binning needs " + std::to_string(need) +
                               " bytes of scratch but the static scratch holds " +
                               std::to_string((size_t)WFPG_BIN_STATIC_SCRATCH_BYTES) +
                               " bytes; use bin_rays with a caller-provided workspace");
    void* scratch = nullptr;
    const int rc0 = scratch_address(&scratch);
    if (rc0 != WFPG_OK) return rc0;
    // bin_rays_impl clears the scratch regions that must start at zero (the
    // per-node counters and flags) on the stream before using them; every
    // other region is fully written before it is read.
    const int rc = wfpg::bin_rays_impl(s, pos, nrm, n, p, sizes, bin_of_ray, ray_order, bin_offset, origin_ray,
                                       bin_cap, n_bins_dev, scratch, (size_t)WFPG_BIN_STATIC_SCRATCH_BYTES,
                                       static_cast<cudaStream_t>(stream));
    if (rc == WFPG_ERR_CUDA)
        return static_fail(rc, std::string("bin_rays_static: ") + cudaGetErrorString(wfpg::take_launch_error()));
    if (rc != WFPG_OK) return static_fail(rc, "bin_rays_static: failed");
    return WFPG_OK;
}

}  // extern "C"
