// extern "C" entry points declared in include/wfpg.h: argument checks,
// handle lifetime, error reporting, and dispatch to the kernels.
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "sort.cuh"
#include "svo.cuh"

namespace wfpg {
int build_svo(const wfpg_scene* scene, int D, cudaStream_t st, wfpg_svo* s, std::string& err);
int accumulate(wfpg_svo* s, const float* pos, const float* wout, const float* L, uint32_t n, cudaStream_t st,
               const uint32_t* n_dev = nullptr);
size_t bin_workspace_bytes(const wfpg_svo* s, uint32_t n, int mode, uint32_t n_sizes);
int bin_rays_impl(const wfpg_svo* s, const float* pos, const float* nrm, uint32_t n, const wfpg_bin_params* p,
                  const uint32_t* sizes, uint32_t* bin_of_ray, uint32_t* ray_order, uint32_t* bin_offset,
                  uint32_t* origin_ray, uint32_t bin_cap, uint32_t* n_bins_dev, void* workspace, size_t ws_bytes,
                  cudaStream_t st, const uint32_t* frame_dev = nullptr);
int guide_build_impl(const wfpg_svo* s, const float* pos, const uint32_t* origin_ray, const uint32_t* n_bins_dev,
                     uint32_t bin_cap, const wfpg_guide_params* p, float* pdf, float* cdf_row, float* cdf_marg,
                     cudaStream_t st, const uint32_t* frame_dev = nullptr);
int guide_fused_impl(const wfpg_svo* s, const float* pos, const float* nrm, const uint32_t* origin_ray,
                     const uint32_t* n_bins_dev, uint32_t bin_cap, const uint32_t* ray_order,
                     const uint32_t* bin_offset, const float* u, float alpha, const wfpg_guide_params* p, float* dir,
                     float* pdf_out, uint32_t n, void* workspace, size_t ws_bytes, cudaStream_t st,
                     const uint32_t* frame_dev = nullptr, const float* eval_dir = nullptr,
                     float* eval_pdf = nullptr);
size_t guide_fused_workspace_bytes(int N, uint32_t n, uint32_t split);
int product_sums_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, float* S,
                      cudaStream_t st);
int product_sample_impl(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                        const uint32_t* bin_of_ray, const float* nrm, const float* u, uint32_t n,
                        const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, uint32_t* cell,
                        cudaStream_t st);
int product_eval_impl(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                      const uint32_t* bin, const float* nrm, const float* dir, uint32_t n, float alpha, float* out,
                      cudaStream_t st, const uint32_t* n_dev = nullptr);
int sample_mix_impl(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                    const uint32_t* n_bins_dev, const uint32_t* bin_of_ray, const float* nrm, const float* u,
                    uint32_t n, const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, cudaStream_t st);
int guide_sample_impl(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                      const uint32_t* bin_of_ray, const float* u, uint32_t n, float* dir, float* pdf_out,
                      uint32_t* cell, cudaStream_t st);
int guide_eval_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* bin, const float* dir, uint32_t n,
                    float* out, cudaStream_t st);
}  // namespace wfpg

using namespace wfpg;

namespace wfpg {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace wfpg

namespace wfpg {
thread_local cudaError_t g_launch_error = cudaSuccess;
int launch_status() {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return WFPG_OK;
    g_launch_error = e;
    return WFPG_ERR_CUDA;
}
cudaError_t take_launch_error() {
    cudaError_t e = g_launch_error;
    g_launch_error = cudaSuccess;
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}
}  // namespace wfpg

namespace {
thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    wfpg::g_launch_error = cudaSuccess;  // a reported failure consumes any remembered launch error
    return code;
}
int cuda_fail(const char* where) {
    const cudaError_t e = wfpg::take_launch_error();
    return fail(WFPG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
bool valid_n(int N) { return N == 8 || N == 16 || N == 32 || N == 64 || N == 128; }
inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }
}  // namespace

namespace wfpg {
// lets entry points defined in other files report through wfpg_last_error()
int set_last_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace wfpg

extern "C" {

const char* wfpg_last_error(void) { return g_last_error.c_str(); }

unsigned long long wfpg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int svo_build(const wfpg_scene* scene, int depth, void* stream, wfpg_svo** out) {
    if (!scene || !out) return fail(WFPG_ERR_INVALID_ARG, "svo_build: null scene or out");
    *out = nullptr;
    if (depth < 1 || depth > WFPG_MAX_DEPTH)
        return fail(WFPG_ERR_INVALID_ARG, "svo_build: depth must be in [1, " + std::to_string(WFPG_MAX_DEPTH) + "]");
    if ((uint64_t)scene->n_quads + scene->n_spheres + scene->n_tris == 0)
        return fail(WFPG_ERR_INVALID_ARG, "svo_build: the scene has no primitive");
    if ((uint64_t)scene->n_quads + scene->n_spheres + scene->n_tris >= (1u << 20))
        return fail(WFPG_ERR_INVALID_ARG, "svo_build: at most 2^20 - 1 primitives");
    if ((scene->n_quads && !scene->quads) || (scene->n_spheres && !scene->spheres) || (scene->n_tris && !scene->tris))
        return fail(WFPG_ERR_INVALID_ARG, "svo_build: null primitive array");
    if (!(scene->size > 0.0f) || !std::isfinite(scene->size))
        return fail(WFPG_ERR_INVALID_ARG, "svo_build: size must be finite and > 0");
    wfpg_svo* s = new wfpg_svo();
    cudaGetDevice(&s->device);
    std::string err;
    const int rc = build_svo(scene, depth, as_stream(stream), s, err);
    if (rc != WFPG_OK) {
        svo_free_arrays(s);
        delete s;
        return fail(rc, "svo_build: " + err);
    }
    *out = s;
    return WFPG_OK;
}

int svo_destroy(wfpg_svo* svo) {
    if (!svo) return WFPG_OK;
    svo_free_arrays(svo);
    delete svo;
    return WFPG_OK;
}

int svo_get_info(const wfpg_svo* s, wfpg_svo_info* out) {
    if (!s || !out) return fail(WFPG_ERR_INVALID_ARG, "svo_get_info: null argument");
    out->depth = s->D;
    out->n_nodes = s->n_nodes;
    out->n_frags = s->n_frags;
    std::memcpy(out->level_off, s->level_off, sizeof(out->level_off));
    out->node = s->node;
    out->parent = s->parent;
    out->normal = reinterpret_cast<const float*>(s->normal);
    out->value = reinterpret_cast<const float*>(s->value);
    return WFPG_OK;
}

int svo_reset_exitance(wfpg_svo* s, void* stream) {
    if (!s) return fail(WFPG_ERR_INVALID_ARG, "svo_reset_exitance: null svo");
    cudaStream_t st = as_stream(stream);
    const size_t n = s->n_nodes;
    if (cudaMemsetAsync(s->acc_sum, 0, 16 * n, st) != cudaSuccess ||
        cudaMemsetAsync(s->acc_cnt, 0, 8 * n, st) != cudaSuccess ||
        cudaMemsetAsync(s->tot_sum, 0, 16 * n, st) != cudaSuccess ||
        cudaMemsetAsync(s->tot_cnt, 0, 8 * n, st) != cudaSuccess ||
        cudaMemsetAsync(s->value, 0, 8 * n, st) != cudaSuccess)
        return cuda_fail("svo_reset_exitance");
    return WFPG_OK;
}

int svo_accumulate(wfpg_svo* s, const float* pos, const float* wout, const float* L, uint32_t n, void* stream) {
    if (!s) return fail(WFPG_ERR_INVALID_ARG, "svo_accumulate: null svo");
    if (n && (!pos || !wout || !L)) return fail(WFPG_ERR_INVALID_ARG, "svo_accumulate: null record array");
    if (accumulate(s, pos, wout, L, n, as_stream(stream)) != WFPG_OK) return cuda_fail("svo_accumulate");
    return WFPG_OK;
}

int bin_rays_workspace_size(const wfpg_svo* s, uint32_t n, const wfpg_bin_params* p, size_t* bytes) {
    if (!s || !p || !bytes) return fail(WFPG_ERR_INVALID_ARG, "bin_rays_workspace_size: null argument");
    if (p->mode != WFPG_BIN_PARTITION_S && p->mode != WFPG_BIN_RUNS)
        return fail(WFPG_ERR_INVALID_ARG, "bin_rays_workspace_size: unknown mode");
    *bytes = bin_workspace_bytes(s, n, p->mode, p->n_sizes);
    return WFPG_OK;
}

int bin_rays(const wfpg_svo* s, const float* pos, const float* nrm, uint32_t n, const wfpg_bin_params* p,
             const uint32_t* sizes, uint32_t* bin_of_ray, uint32_t* ray_order, uint32_t* bin_offset,
             uint32_t* origin_ray, uint32_t bin_cap, uint32_t* n_bins_dev, void* workspace, size_t ws_bytes,
             void* stream) {
    if (!s || !p) return fail(WFPG_ERR_INVALID_ARG, "bin_rays: null svo or params");
    if (p->mode != WFPG_BIN_PARTITION_S && p->mode != WFPG_BIN_RUNS)
        return fail(WFPG_ERR_INVALID_ARG, "bin_rays: unknown mode");
    if (n >= 0x80000000u) return fail(WFPG_ERR_INVALID_ARG, "bin_rays: at most 2^31 - 1 rays");
    if (n && (!pos || !bin_of_ray || !ray_order)) return fail(WFPG_ERR_INVALID_ARG, "bin_rays: null ray array");
    if (!bin_offset || !n_bins_dev || (bin_cap && !origin_ray))
        return fail(WFPG_ERR_INVALID_ARG, "bin_rays: null bin array");
    if (p->mode == WFPG_BIN_RUNS) {
        if (n && !nrm) return fail(WFPG_ERR_INVALID_ARG, "bin_rays: RUNS mode needs nrm");
        if (p->n_sizes == 0 || !sizes) return fail(WFPG_ERR_INVALID_ARG, "bin_rays: RUNS mode needs sizes");
        if (p->n_sizes > bin_cap)
            return fail(WFPG_ERR_CAPACITY, "bin_rays: n_sizes exceeds bin_cap");
    }
    const size_t need = bin_workspace_bytes(s, n, p->mode, p->n_sizes);
    if (!workspace || ws_bytes < need)
        return fail(WFPG_ERR_INVALID_ARG, "bin_rays: workspace smaller than bin_rays_workspace_size() = " +
                                              std::to_string(need) + " bytes");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return fail(WFPG_ERR_INVALID_ARG, "bin_rays: workspace must be 256-byte aligned");
    const int rc = bin_rays_impl(s, pos, nrm, n, p, sizes, bin_of_ray, ray_order, bin_offset, origin_ray, bin_cap,
                                 n_bins_dev, workspace, ws_bytes, as_stream(stream));
    if (rc == WFPG_ERR_CUDA) return cuda_fail("bin_rays");
    if (rc != WFPG_OK) return fail(rc, "bin_rays: failed");
    return WFPG_OK;
}

int guide_build_pdf(const wfpg_svo* s, const float* pos, const uint32_t* origin_ray, const uint32_t* n_bins_dev,
                    uint32_t bin_cap, const wfpg_guide_params* p, float* pdf, float* cdf_row, float* cdf_marg,
                    void* stream) {
    if (!s || !p) return fail(WFPG_ERR_INVALID_ARG, "guide_build_pdf: null svo or params");
    if (!valid_n(p->N)) return fail(WFPG_ERR_INVALID_ARG, "guide_build_pdf: N must be 8, 16, 32, 64 or 128");
    if (p->parts != 0 && p->parts != 1 && p->parts != 2 && p->parts != 4 && p->parts != 8)
        return fail(WFPG_ERR_INVALID_ARG, "guide_build_pdf: parts must be 0, 1, 2, 4 or 8");
    if (!(p->eps >= 0.0f)) return fail(WFPG_ERR_INVALID_ARG, "guide_build_pdf: eps must be >= 0");
    if (p->block != 0 && p->block != 64 && p->block != 128 && p->block != 256)
        return fail(WFPG_ERR_INVALID_ARG, "guide_build_pdf: block must be 0, 64, 128 or 256");
    if (bin_cap && (!pos || !pdf || !cdf_row || !cdf_marg))
        return fail(WFPG_ERR_INVALID_ARG, "guide_build_pdf: null array");
    const int rc = guide_build_impl(s, pos, origin_ray, n_bins_dev, bin_cap, p, pdf, cdf_row, cdf_marg,
                                    as_stream(stream));
    if (rc == WFPG_ERR_INVALID_ARG)
        return fail(rc, "guide_build_pdf: the field of side " + std::to_string(p->N) +
                            " does not fit in shared memory with this block size");
    if (rc != WFPG_OK) return cuda_fail("guide_build_pdf");
    return WFPG_OK;
}

int guide_build_sample_workspace_size(int N, uint32_t n, uint32_t split, size_t* bytes) {
    if (!bytes) return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample_workspace_size: null bytes");
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample_workspace_size: bad N");
    *bytes = guide_fused_workspace_bytes(N, n, split);
    return WFPG_OK;
}

int guide_build_sample(const wfpg_svo* s, const float* pos, const float* nrm, const uint32_t* origin_ray,
                       const uint32_t* n_bins_dev, uint32_t bin_cap, const uint32_t* ray_order,
                       const uint32_t* bin_offset, const float* u, uint32_t n, float alpha,
                       const wfpg_guide_params* p, float* dir, float* pdf_out, void* workspace, size_t ws_bytes,
                       void* stream) {
    if (!s || !p) return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample: null svo or params");
    if (!valid_n(p->N)) return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample: N must be 8, 16, 32, 64 or 128");
    if (!(p->eps >= 0.0f)) return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample: eps must be >= 0");
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample: alpha in [0, 1]");
    if (p->block != 0 && p->block != 64 && p->block != 128 && p->block != 256)
        return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample: block must be 0, 64, 128 or 256");
    if (bin_cap && (!pos || !nrm || !ray_order || !bin_offset || !u || !dir || !pdf_out))
        return fail(WFPG_ERR_INVALID_ARG, "guide_build_sample: null array");
    if (ws_bytes < guide_fused_workspace_bytes(p->N, n, p->split) || (ws_bytes && !workspace))
        return fail(WFPG_ERR_CAPACITY, "guide_build_sample: workspace too small");
    const int rc = guide_fused_impl(s, pos, nrm, origin_ray, n_bins_dev, bin_cap, ray_order, bin_offset, u, alpha, p,
                                    dir, pdf_out, n, workspace, ws_bytes, as_stream(stream));
    if (rc == WFPG_ERR_INVALID_ARG)
        return fail(rc, "guide_build_sample: the field does not fit in shared memory with this block size");
    if (rc != WFPG_OK) return cuda_fail("guide_build_sample");
    return WFPG_OK;
}

int guide_product_sums(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, float* S,
                       void* stream) {
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_product_sums: N must be 8, 16, 32, 64 or 128");
    if (bin_cap && (!pdf || !S)) return fail(WFPG_ERR_INVALID_ARG, "guide_product_sums: null array");
    if (product_sums_impl(pdf, N, bin_cap, n_bins_dev, S, as_stream(stream)) != WFPG_OK)
        return cuda_fail("guide_product_sums");
    return WFPG_OK;
}

int guide_product_sample(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                         const uint32_t* bin_of_ray, const float* nrm, const float* u, uint32_t n,
                         const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, uint32_t* cell,
                         void* stream) {
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_product_sample: N must be 8, 16, 32, 64 or 128");
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(WFPG_ERR_INVALID_ARG, "guide_product_sample: alpha in [0, 1]");
    if (n && (!bin_of_ray || !nrm || !u || !dir || !pdf_out || (bin_cap && (!pdf || !S))))
        return fail(WFPG_ERR_INVALID_ARG, "guide_product_sample: null array");
    if (product_sample_impl(pdf, S, N, bin_cap, n_bins_dev, bin_of_ray, nrm, u, n, n_dev, alpha, dir, pdf_out, cell,
                            as_stream(stream)) != WFPG_OK)
        return cuda_fail("guide_product_sample");
    return WFPG_OK;
}

int guide_product_eval(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                       const uint32_t* bin, const float* nrm, const float* dir, uint32_t n, float alpha, float* out,
                       void* stream) {
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_product_eval: N must be 8, 16, 32, 64 or 128");
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(WFPG_ERR_INVALID_ARG, "guide_product_eval: alpha in [0, 1]");
    if (n && (!bin || !nrm || !dir || !out || (bin_cap && (!pdf || !S))))
        return fail(WFPG_ERR_INVALID_ARG, "guide_product_eval: null array");
    if (product_eval_impl(pdf, S, N, bin_cap, n_bins_dev, bin, nrm, dir, n, alpha, out, as_stream(stream)) != WFPG_OK)
        return cuda_fail("guide_product_eval");
    return WFPG_OK;
}

int guide_sample_mix(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                     const uint32_t* n_bins_dev, const uint32_t* bin_of_ray, const float* nrm, const float* u,
                     uint32_t n, const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, void* stream) {
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_sample_mix: N must be 8, 16, 32, 64 or 128");
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(WFPG_ERR_INVALID_ARG, "guide_sample_mix: alpha in [0, 1]");
    if (n && (!bin_of_ray || !nrm || !u || !dir || !pdf_out || (bin_cap && (!pdf || !cdf_row || !cdf_marg))))
        return fail(WFPG_ERR_INVALID_ARG, "guide_sample_mix: null array");
    if (sample_mix_impl(pdf, cdf_row, cdf_marg, N, bin_cap, n_bins_dev, bin_of_ray, nrm, u, n, n_dev, alpha, dir,
                        pdf_out, as_stream(stream)) != WFPG_OK)
        return cuda_fail("guide_sample_mix");
    return WFPG_OK;
}

int guide_sample(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                 const uint32_t* bin_of_ray, const float* u, uint32_t n, float* dir, float* pdf_out, uint32_t* cell,
                 void* stream) {
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_sample: N must be 8, 16, 32, 64 or 128");
    if (n && (!pdf || !cdf_row || !cdf_marg || !bin_of_ray || !u || !dir || !pdf_out || !cell))
        return fail(WFPG_ERR_INVALID_ARG, "guide_sample: null array");
    if (reinterpret_cast<uintptr_t>(u) & 7u) return fail(WFPG_ERR_INVALID_ARG, "guide_sample: u must be 8-byte aligned");
    if (guide_sample_impl(pdf, cdf_row, cdf_marg, N, bin_cap, bin_of_ray, u, n, dir, pdf_out, cell,
                          as_stream(stream)) != WFPG_OK)
        return cuda_fail("guide_sample");
    return WFPG_OK;
}

int guide_eval_pdf(const float* pdf, int N, uint32_t bin_cap, const uint32_t* bin, const float* dir, uint32_t n,
                   float* out, void* stream) {
    if (!valid_n(N)) return fail(WFPG_ERR_INVALID_ARG, "guide_eval_pdf: N must be 8, 16, 32, 64 or 128");
    if (n && (!pdf || !bin || !dir || !out)) return fail(WFPG_ERR_INVALID_ARG, "guide_eval_pdf: null array");
    if (guide_eval_impl(pdf, N, bin_cap, bin, dir, n, out, as_stream(stream)) != WFPG_OK)
        return cuda_fail("guide_eval_pdf");
    return WFPG_OK;
}

int svo_export(const wfpg_svo* s, uint64_t* key, uint32_t* first_child, uint8_t* child_mask, uint32_t* parent,
               float* normal3, uint32_t* leaf_count, uint32_t* frag_off, uint32_t* frag_prim, void* stream) {
    if (!s) return fail(WFPG_ERR_INVALID_ARG, "svo_export: null svo");
    cudaStream_t st = as_stream(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail("svo_export");
    const size_t n = s->n_nodes;
    std::vector<Node> nodes(n);
    std::vector<float4> nrm(n);
    bool ok = cudaMemcpy(nodes.data(), s->node, n * sizeof(Node), cudaMemcpyDeviceToHost) == cudaSuccess &&
              cudaMemcpy(nrm.data(), s->normal, n * sizeof(float4), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && key) ok = cudaMemcpy(key, s->key, n * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && parent) ok = cudaMemcpy(parent, s->parent, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && leaf_count) ok = cudaMemcpy(leaf_count, s->leaf_count, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    const size_t nl = s->level_off[s->D + 1] - s->level_off[s->D];
    if (ok && frag_off) ok = cudaMemcpy(frag_off, s->frag_off, (nl + 1) * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && frag_prim) ok = cudaMemcpy(frag_prim, s->frag_prim, (size_t)s->n_frags * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return cuda_fail("svo_export");
    for (size_t i = 0; i < n; ++i) {
        if (first_child) first_child[i] = nodes[i].first_child;
        if (child_mask) child_mask[i] = (uint8_t)nodes[i].mask;
        if (normal3) {
            normal3[3 * i + 0] = nrm[i].x;
            normal3[3 * i + 1] = nrm[i].y;
            normal3[3 * i + 2] = nrm[i].z;
        }
    }
    return WFPG_OK;
}

int svo_export_exitance(const wfpg_svo* s, uint64_t* acc_sum, uint32_t* acc_cnt, uint64_t* tot_sum, uint32_t* tot_cnt,
                        float* value, void* stream) {
    if (!s) return fail(WFPG_ERR_INVALID_ARG, "svo_export_exitance: null svo");
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return cuda_fail("svo_export_exitance");
    const size_t n = 2 * (size_t)s->n_nodes;
    bool ok = true;
    if (acc_sum) ok = ok && cudaMemcpy(acc_sum, s->acc_sum, n * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (acc_cnt) ok = ok && cudaMemcpy(acc_cnt, s->acc_cnt, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (tot_sum) ok = ok && cudaMemcpy(tot_sum, s->tot_sum, n * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (tot_cnt) ok = ok && cudaMemcpy(tot_cnt, s->tot_cnt, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (value) ok = ok && cudaMemcpy(value, s->value, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return cuda_fail("svo_export_exitance");
    return WFPG_OK;
}

int wfpg_svo_status(wfpg_svo* s, uint32_t* flags, int clear, void* stream) {
    if (!s || !flags) return fail(WFPG_ERR_INVALID_ARG, "wfpg_svo_status: null argument");
    cudaStream_t st = as_stream(stream);
    if (cudaMemcpyAsync(flags, s->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_fail("wfpg_svo_status");
    if (clear && (cudaMemsetAsync(s->status, 0, 4, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess))
        return cuda_fail("wfpg_svo_status");
    return WFPG_OK;
}

}  // extern "C"
