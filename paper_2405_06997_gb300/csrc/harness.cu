// Renderer-side helper for measuring the guiding (not part of the paper's
// method): closest-hit ray casting against the scenes' quads, spheres and
// triangles, so that guided estimators can be evaluated against the scene's
// true incident radiance.
#include <string>

#include "cast.cuh"
#include "svo.cuh"

namespace wfpg {

__global__ void __launch_bounds__(256) k_cast(Prims S, const float* __restrict__ o, const float* __restrict__ d, uint32_t n,
                                              float tmin, float* __restrict__ t_out, uint32_t* __restrict__ prim_out,
                                              float* __restrict__ nrm_out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ox = o[3 * (size_t)i], oy = o[3 * (size_t)i + 1], oz = o[3 * (size_t)i + 2];
    const float dx = d[3 * (size_t)i], dy = d[3 * (size_t)i + 1], dz = d[3 * (size_t)i + 2];
    const Hit h = cast_closest(S, ox, oy, oz, dx, dy, dz, tmin);
    t_out[i] = h.t;
    prim_out[i] = h.prim;
    if (nrm_out) {
        const float3 nn = hit_normal(S, h, ox, oy, oz, dx, dy, dz);
        nrm_out[3 * (size_t)i] = nn.x;
        nrm_out[3 * (size_t)i + 1] = nn.y;
        nrm_out[3 * (size_t)i + 2] = nn.z;
    }
}

__global__ void __launch_bounds__(256) k_cast_svo(SvoCast V, Prims S, const float* __restrict__ o,
                                                  const float* __restrict__ d, uint32_t n, float tmin,
                                                  float* __restrict__ t_out, uint32_t* __restrict__ prim_out,
                                                  float* __restrict__ nrm_out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ox = o[3 * (size_t)i], oy = o[3 * (size_t)i + 1], oz = o[3 * (size_t)i + 2];
    const float dx = d[3 * (size_t)i], dy = d[3 * (size_t)i + 1], dz = d[3 * (size_t)i + 2];
    const Hit h = cast_svo(V, S, ox, oy, oz, dx, dy, dz, tmin);
    t_out[i] = h.t;
    prim_out[i] = h.prim;
    if (nrm_out) {
        const float3 nn = hit_normal(S, h, ox, oy, oz, dx, dy, dz);
        nrm_out[3 * (size_t)i] = nn.x;
        nrm_out[3 * (size_t)i + 1] = nn.y;
        nrm_out[3 * (size_t)i + 2] = nn.z;
    }
}

SvoCast svo_cast_view(const wfpg_svo* s) {
    SvoCast V;
    V.node = s->node;
    V.frag_off = s->frag_off;
    V.frag_prim = s->frag_prim;
    V.leaf_off = s->level_off[s->D];
    V.D = s->D;
    for (int a = 0; a < 3; ++a) V.lo[a] = s->lo[a];
    V.scale = s->scale;
    return V;
}

int set_last_error(int code, const std::string& msg);

}  // namespace wfpg

extern "C" int wfpg_cast_rays(const wfpg_scene* scene, const float* o, const float* d, uint32_t n, float tmin,
                              float* t_out, uint32_t* prim_out, float* nrm_out, void* stream) {
    if (!scene || (n && (!o || !d || !t_out || !prim_out)))
        return wfpg::set_last_error(WFPG_ERR_INVALID_ARG, "wfpg_cast_rays: null argument");
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(wfpg::k_cast, wfpg::div_up(n, 256), 256, 0, static_cast<cudaStream_t>(stream),
                wfpg::prims_of(*scene), o, d, n, tmin, t_out, prim_out, nrm_out);
    if (cudaGetLastError() != cudaSuccess) return wfpg::set_last_error(WFPG_ERR_CUDA, "wfpg_cast_rays: launch failed");
    return WFPG_OK;
}

extern "C" int wfpg_cast_rays_svo(const wfpg_svo* svo, const wfpg_scene* scene, const float* o, const float* d,
                                  uint32_t n, float tmin, float* t_out, uint32_t* prim_out, float* nrm_out,
                                  void* stream) {
    if (!svo || !scene || (n && (!o || !d || !t_out || !prim_out)))
        return wfpg::set_last_error(WFPG_ERR_INVALID_ARG, "wfpg_cast_rays_svo: null argument");
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(wfpg::k_cast_svo, wfpg::div_up(n, 256), 256, 0, static_cast<cudaStream_t>(stream),
                wfpg::svo_cast_view(svo), wfpg::prims_of(*scene), o, d, n, tmin, t_out, prim_out, nrm_out);
    if (cudaGetLastError() != cudaSuccess)
        return wfpg::set_last_error(WFPG_ERR_CUDA, "wfpg_cast_rays_svo: launch failed");
    return WFPG_OK;
}
