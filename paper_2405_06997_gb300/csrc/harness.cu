// Renderer-side helper for measuring the guiding (not part of the paper's
// method): closest-hit ray casting against the procedural scenes' analytic
// quads and spheres, so that guided estimators can be evaluated against the
// scene's true incident radiance.
#include <string>

#include "common.cuh"

namespace wfpg {

__global__ void __launch_bounds__(256) k_cast(const float* __restrict__ quads, uint32_t nq,
                                              const float* __restrict__ spheres, uint32_t ns,
                                              const float* __restrict__ o, const float* __restrict__ d, uint32_t n,
                                              float tmin, float* __restrict__ t_out, uint32_t* __restrict__ prim_out,
                                              float* __restrict__ nrm_out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ox = o[3 * (size_t)i], oy = o[3 * (size_t)i + 1], oz = o[3 * (size_t)i + 2];
    const float dx = d[3 * (size_t)i], dy = d[3 * (size_t)i + 1], dz = d[3 * (size_t)i + 2];
    const float oo[3] = {ox, oy, oz}, dd[3] = {dx, dy, dz};
    float best = __int_as_float(0x7f800000);
    uint32_t bp = kNone;
    for (uint32_t q = 0; q < nq; ++q) {
        const float* Q = quads + 8 * (size_t)q;
        const int a = (int)Q[0], b = (a + 1) % 3, c = (a + 2) % 3;
        if (dd[a] == 0.0f) continue;
        const float t = (Q[1] - oo[a]) / dd[a];
        if (!(t > tmin) || t >= best) continue;
        const float pb = oo[b] + t * dd[b], pc = oo[c] + t * dd[c];
        if (pb >= Q[2] && pb <= Q[3] && pc >= Q[4] && pc <= Q[5]) {
            best = t;
            bp = q;
        }
    }
    for (uint32_t s = 0; s < ns; ++s) {
        const float* S = spheres + 4 * (size_t)s;
        const float cx = ox - S[0], cy = oy - S[1], cz = oz - S[2];
        const float bq = dx * cx + dy * cy + dz * cz;
        const float cq = cx * cx + cy * cy + cz * cz - S[3] * S[3];
        const float disc = bq * bq - cq;
        if (disc < 0.0f) continue;
        const float sq = sqrtf(disc);
        float t = -bq - sq;
        if (!(t > tmin)) t = -bq + sq;
        if (t > tmin && t < best) {
            best = t;
            bp = nq + s;
        }
    }
    t_out[i] = bp == kNone ? -1.0f : best;
    prim_out[i] = bp;
    if (nrm_out) {
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (bp != kNone && bp < nq) {
            const float* Q = quads + 8 * (size_t)bp;
            const int a = (int)Q[0];
            (a == 0 ? nx : (a == 1 ? ny : nz)) = Q[6];
        } else if (bp != kNone) {
            const float* S = spheres + 4 * (size_t)(bp - nq);
            nx = (ox + best * dx - S[0]) / S[3];
            ny = (oy + best * dy - S[1]) / S[3];
            nz = (oz + best * dz - S[2]) / S[3];
        }
        if (nx * dx + ny * dy + nz * dz > 0.0f) {  // face the incoming ray
            nx = -nx;
            ny = -ny;
            nz = -nz;
        }
        nrm_out[3 * (size_t)i] = nx;
        nrm_out[3 * (size_t)i + 1] = ny;
        nrm_out[3 * (size_t)i + 2] = nz;
    }
}

int set_last_error(int code, const std::string& msg);

}  // namespace wfpg

extern "C" int wfpg_cast_rays(const wfpg_scene* scene, const float* o, const float* d, uint32_t n, float tmin,
                              float* t_out, uint32_t* prim_out, float* nrm_out, void* stream) {
    if (!scene || (n && (!o || !d || !t_out || !prim_out)))
        return wfpg::set_last_error(WFPG_ERR_INVALID_ARG, "wfpg_cast_rays: null argument");
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(wfpg::k_cast, wfpg::div_up(n, 256), 256, 0, static_cast<cudaStream_t>(stream), scene->quads,
                scene->n_quads, scene->spheres, scene->n_spheres, o, d, n, tmin, t_out, prim_out, nrm_out);
    if (cudaGetLastError() != cudaSuccess) return wfpg::set_last_error(WFPG_ERR_CUDA, "wfpg_cast_rays: launch failed");
    return WFPG_OK;
}
