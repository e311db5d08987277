// Batched wavefront frame: Alg. 1 for every pixel of a pinhole camera with
// no host round trip, captured once as a CUDA graph and replayed per frame.
//
// Per depth the live paths sit in a compact queue (structure of arrays, in
// pixel order: compaction is an exclusive scan, so every run is
// deterministic); Partition-S and the fused GuideRays launch read the queue
// length from device memory, so the same launches serve every depth and
// every frame.  The path history (throughput, emission, position and
// direction toward the previous vertex, per vertex) is kept for Eq. 5, which
// runs once per frame after the last depth (UpdateExitance in Alg. 1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cast.cuh"
#include "common.cuh"
#include "sort.cuh"
#include "svo.cuh"

namespace wfpg {

int set_last_error(int code, const std::string& msg);
void note_launches(long long n);
int bin_rays_impl(const wfpg_svo* s, const float* pos, const float* nrm, uint32_t n, const wfpg_bin_params* p,
                  const uint32_t* sizes, uint32_t* bin_of_ray, uint32_t* ray_order, uint32_t* bin_offset,
                  uint32_t* origin_ray, uint32_t bin_cap, uint32_t* n_bins_dev, void* workspace, size_t ws_bytes,
                  cudaStream_t st, const uint32_t* frame_dev);
size_t bin_workspace_bytes(const wfpg_svo* s, uint32_t n, int mode, uint32_t n_sizes);
int guide_fused_impl(const wfpg_svo* s, const float* pos, const float* nrm, const uint32_t* origin_ray,
                     const uint32_t* n_bins_dev, uint32_t bin_cap, const uint32_t* ray_order,
                     const uint32_t* bin_offset, const float* u, float alpha, const wfpg_guide_params* p, float* dir,
                     float* pdf_out, uint32_t n, void* workspace, size_t ws_bytes, cudaStream_t st,
                     const uint32_t* frame_dev, const float* eval_dir, float* eval_pdf);
size_t guide_fused_workspace_bytes(int N, uint32_t n, uint32_t split);
int accumulate(wfpg_svo* s, const float* pos, const float* wout, const float* L, uint32_t n, cudaStream_t st,
               const uint32_t* n_dev);
int sample_mix_impl(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                    const uint32_t* n_bins_dev, const uint32_t* bin_of_ray, const float* nrm, const float* u,
                    uint32_t n, const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, cudaStream_t st);
SvoCast svo_cast_view(const wfpg_svo* s);
int product_eval_impl(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                      const uint32_t* bin, const float* nrm, const float* dir, uint32_t n, float alpha, float* out,
                      cudaStream_t st, const uint32_t* n_dev);
int mix_eval_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, const uint32_t* bin_of_ray,
                  const float* nrm, const float* dir, uint32_t n, const uint32_t* n_dev, float alpha, float* out,
                  cudaStream_t st);
int guide_build_impl(const wfpg_svo* s, const float* pos, const uint32_t* origin_ray, const uint32_t* n_bins_dev,
                     uint32_t bin_cap, const wfpg_guide_params* p, float* pdf, float* cdf_row, float* cdf_marg,
                     cudaStream_t st, const uint32_t* frame_dev);
int product_sums_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, float* S,
                      cudaStream_t st);
int product_sample_impl(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                        const uint32_t* bin_of_ray, const float* nrm, const float* u, uint32_t n,
                        const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, uint32_t* cell,
                        cudaStream_t st);
uint32_t mlp_max_batch(const wfpg_mlp* m);

constexpr uint64_t kPathPurpose = 2;  // per-path uniforms (0: origins, 1: jitter)
constexpr uint32_t kPathStride = 8;   // uniforms per depth: direction 0-1, mixture 2, roulette 3, light 4-6
constexpr uint32_t kDepthStride = 16; // random-stream frame index = frame * 16 + depth
constexpr float kInvPi = 0.31830988618379067f;

// one queue of live paths (or the staging copy the shading writes)
struct Queue {
    uint32_t* path;
    float* pos;  // xyz
    float* nrm;  // xyz, facing the incoming ray
    float* T;    // throughput of the continuation (Russian roulette included)
    float* alb;  // albedo at the vertex
    float* u;    // xyz uniforms of the next direction (queues only)
};

struct FrameView {
    Prims pr;                     // the scene's quads, spheres and triangles
    const float* emission;
    const float* albedo;
    uint32_t P, W, H;
    float eye[3], fwd[3], right[3], up[3];  // right and up scaled by the image-plane half extents
    const float* probe_pos;                   // probe mode: points [H][3] (null: pinhole)
    uint32_t probe_n;                         // probe mode: side of the octahedral grid (W = probe_n^2)
    int max_depth, rr_depth;
    uint64_t pseed;
    float offset;  // origin offset along the normal for continuation rays
    SvoCast sv;
    int svo_cast;  // 1: closest hits by the SVO walk, 0: every primitive
    float* vT;
    float* vLe;
    float* vpos;
    float* vwo;
    uint32_t* nv;
    double* img_sum;
    double* img_sq;
    double* img_wsum;  // sum of h(i) x estimate
    // next-event estimation (0 lights: off)
    int nee;
    uint32_t n_lights;
    const uint32_t* light_prim;   // emissive primitives
    const float* light_cdf;       // inclusive power CDF over them (last = 1)
    const float* prim_pmf;        // per primitive: its selection probability (0 if not a light)
    const float* prim_area;       // per primitive: area
    float* nee_dir;               // per queue slot: direction to the light sample
    float* nee_l;                 // per queue slot: f cos Le / p_light (0: no unoccluded sample)
    float* nee_pl;                // per queue slot: light sample density (solid angle)
    float* nee_pm;                // per queue slot: the mixture's density at nee_dir
    float* vNee;                  // per vertex: MIS-weighted light sample per unit T(p_k)
    float* vLw;                   // per vertex: its emission as the previous vertex sees it (MIS-weighted)
    double* wsum;      // sum of h(i)
    int combine;
    uint32_t* counters;  // [0 .. max_depth - 1]: paths per depth; [WFPG_FRAME_MAX_DEPTH + 1]: records
    uint32_t* fidx;      // [0 .. max_depth]: random-stream frame index per depth
    uint32_t* frame_counter;
    unsigned long long* frames_run;
    unsigned long long* guided;
};

__device__ __forceinline__ float path_uniform(const FrameView& F, uint32_t path, uint32_t counter) {
    return uniform01(F.pseed, ((uint64_t)F.fidx[0] << 32) | path, counter);
}

// Eq. 7's frame weight h(i), i = 1, 2, ... (PT first weighs every frame 1; its
// first frame runs unguided)
__device__ __forceinline__ double combine_weight(int combine, unsigned long long i) {
    switch (combine) {
        case 1: return (double)(i < 5 ? i : 5);
        case 2: return (double)(i < 5 ? i * i : 25);
        case 3: return i == 1 ? 1.0 : 2.0;
        case 4: return i == 1 ? 0.0 : 1.0;
        default: return 1.0;
    }
}

__global__ void k_frame_begin(FrameView F) {
    const uint32_t fc = *F.frame_counter;
    for (int k = threadIdx.x; k <= F.max_depth; k += blockDim.x) F.fidx[k] = fc * kDepthStride + k;
    for (int k = threadIdx.x; k <= WFPG_FRAME_MAX_DEPTH + 1; k += blockDim.x) F.counters[k] = 0;
}

__device__ __forceinline__ Hit frame_cast(const FrameView& F, float ox, float oy, float oz, float dx, float dy,
                                          float dz) {
    return F.svo_cast ? cast_svo(F.sv, F.pr, ox, oy, oz, dx, dy, dz, 0.0f)
                      : cast_closest(F.pr, ox, oy, oz, dx, dy, dz, 0.0f);
}

// survival test at 1-based vertex v (>= rr_depth): min(0.95, albedo)
__device__ __forceinline__ bool roulette(const FrameView& F, uint32_t path, int v, float alb, float* T) {
    if (v < F.rr_depth) return true;
    const float q = fminf(0.95f, alb);
    if (path_uniform(F, path, kPathStride * (uint32_t)(v - 1) + 3u) >= q) return false;
    *T = *T / q;
    return true;
}

__device__ __forceinline__ void store3(float* a, size_t i, float x, float y, float z) {
    a[3 * i] = x;
    a[3 * i + 1] = y;
    a[3 * i + 2] = z;
}

// primary rays through pixel centres, their closest hits = vertex 1
__global__ void __launch_bounds__(256) k_camera(FrameView F, Queue S, uint32_t* __restrict__ flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.P) return;
    const uint32_t x = i % F.W, y = i / F.W;
    float ex = F.eye[0], ey = F.eye[1], ez = F.eye[2], dx, dy, dz;
    if (F.probe_pos) {  // a uniform direction inside octahedral cell x around probe y
        const uint32_t c0 = kPathStride * WFPG_FRAME_MAX_DEPTH;
        const float tn = 2.0f / (float)F.probe_n;
        const float su = ((float)(x % F.probe_n) + path_uniform(F, i, c0)) * tn - 1.0f;
        const float sv = ((float)(x / F.probe_n) + path_uniform(F, i, c0 + 1)) * tn - 1.0f;
        const float3 d = octa_to_dir(fminf(su, 1.0f), fminf(sv, 1.0f));
        dx = d.x;
        dy = d.y;
        dz = d.z;
        ex = F.probe_pos[3 * (size_t)y];
        ey = F.probe_pos[3 * (size_t)y + 1];
        ez = F.probe_pos[3 * (size_t)y + 2];
    } else {
        const float px = ((float)x + 0.5f) / (float)F.W * 2.0f - 1.0f;
        const float py = 1.0f - ((float)y + 0.5f) / (float)F.H * 2.0f;
        dx = F.fwd[0] + px * F.right[0] + py * F.up[0];
        dy = F.fwd[1] + px * F.right[1] + py * F.up[1];
        dz = F.fwd[2] + px * F.right[2] + py * F.up[2];
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv;
        dy *= inv;
        dz *= inv;
    }
    const Hit h = frame_cast(F, ex, ey, ez, dx, dy, dz);
    uint32_t flag = 0;
    F.nv[i] = 0;
    if (h.prim != kNone) {
        const float hx = ex + h.t * dx, hy = ey + h.t * dy, hz = ez + h.t * dz;
        const float3 n = hit_normal(F.pr, h, ex, ey, ez, dx, dy, dz);
        const float a = F.albedo[h.prim];
        F.vT[i] = 1.0f;
        F.vLe[i] = F.emission[h.prim];  // seen by the camera: no other strategy to weigh against
        if (F.nee) {
            F.vNee[i] = 0.0f;
            F.vLw[i] = F.vLe[i];
        }
        store3(F.vpos, i, hx, hy, hz);
        store3(F.vwo, i, -dx, -dy, -dz);
        F.nv[i] = 1;
        float T = 1.0f;
        if (a > 0.0f && F.max_depth >= 1 && roulette(F, i, 1, a, &T)) {
            S.path[i] = i;
            store3(S.pos, i, hx, hy, hz);
            store3(S.nrm, i, n.x, n.y, n.z);
            S.T[i] = T;
            S.alb[i] = a;
            flag = 1;
        }
    }
    flags[i] = flag;
}

// staging slot i -> queue slot offs[i] for the survivors; draws the uniforms of depth k
__global__ void __launch_bounds__(256) k_compact(FrameView F, Queue S, Queue Q, const uint32_t* __restrict__ flags,
                                                 const uint32_t* __restrict__ offs, int k) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.P || !flags[i]) return;
    const uint32_t j = offs[i];
    const uint32_t path = S.path[i];
    Q.path[j] = path;
    store3(Q.pos, j, S.pos[3 * (size_t)i], S.pos[3 * (size_t)i + 1], S.pos[3 * (size_t)i + 2]);
    store3(Q.nrm, j, S.nrm[3 * (size_t)i], S.nrm[3 * (size_t)i + 1], S.nrm[3 * (size_t)i + 2]);
    Q.T[j] = S.T[i];
    Q.alb[j] = S.alb[i];
    const uint32_t c = kPathStride * (uint32_t)k;
    store3(Q.u, j, path_uniform(F, path, c), path_uniform(F, path, c + 1), path_uniform(F, path, c + 2));
}

// light-sample density (solid angle) of reaching emissive primitive `prim` at
// distance t along a direction whose cosine with the light's normal is cl
__device__ __forceinline__ float light_pdf(const FrameView& F, uint32_t prim, float t, float cl) {
    const float pmf = F.prim_pmf[prim];
    if (!(pmf > 0.0f) || !(cl > 0.0f)) return 0.0f;
    return pmf * t * t / (F.prim_area[prim] * cl);
}

// geometric normal of a primitive at point (x, y, z) (unnormalised side)
__device__ __forceinline__ float3 prim_normal(const FrameView& F, uint32_t prim, float x, float y, float z) {
    if (prim < F.pr.nq) {
        const float* Q = F.pr.quads + 8 * (size_t)prim;
        const int a = (int)Q[0];
        return make_float3(a == 0 ? 1.0f : 0.0f, a == 1 ? 1.0f : 0.0f, a == 2 ? 1.0f : 0.0f);
    }
    if (prim >= F.pr.nq + F.pr.ns) {
        const float3 c = tri_cross(F.pr.tris + 9 * (size_t)(prim - F.pr.nq - F.pr.ns));
        const float inv = 1.0f / sqrtf(dot3(c, c));
        return make_float3(c.x * inv, c.y * inv, c.z * inv);
    }
    const float* Sp = F.pr.spheres + 4 * (size_t)(prim - F.pr.nq);
    return make_float3((x - Sp[0]) / Sp[3], (y - Sp[1]) / Sp[3], (z - Sp[2]) / Sp[3]);
}

// next-event estimation at the queue's vertices: an emissive primitive by
// power, a uniform point on it, a shadow ray; Lambertian f cos Le / p_light
__global__ void __launch_bounds__(256) k_nee(FrameView F, Queue Q, int k) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= F.counters[k]) return;
    const uint32_t path = Q.path[s];
    const uint32_t c0 = kPathStride * (uint32_t)k + 4u;
    const float us = path_uniform(F, path, c0), ua = path_uniform(F, path, c0 + 1), ub = path_uniform(F, path, c0 + 2);
    // the first light whose inclusive power CDF exceeds us (bisection; the last CDF entry is 1)
    uint32_t lo = 0, hi = F.n_lights - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (F.light_cdf[mid] > us) hi = mid;
        else lo = mid + 1;
    }
    const uint32_t l = lo;
    const uint32_t prim = F.light_prim[l];
    float y[3];
    if (prim < F.pr.nq) {
        const float* Qd = F.pr.quads + 8 * (size_t)prim;
        const int a = (int)Qd[0], b = (a + 1) % 3, c = (a + 2) % 3;
        y[a] = Qd[1];
        y[b] = Qd[2] + ua * (Qd[3] - Qd[2]);
        y[c] = Qd[4] + ub * (Qd[5] - Qd[4]);
    } else if (prim >= F.pr.nq + F.pr.ns) {  // uniform on the triangle: barycentrics (1 - sqrt(ua), ub sqrt(ua))
        const float* T = F.pr.tris + 9 * (size_t)(prim - F.pr.nq - F.pr.ns);
        const float su = sqrtf(ua), b0 = 1.0f - su, b1 = ub * su, b2 = 1.0f - b0 - b1;
        for (int a = 0; a < 3; ++a) y[a] = b0 * T[a] + b1 * T[3 + a] + b2 * T[6 + a];
    } else {
        const float* Sp = F.pr.spheres + 4 * (size_t)(prim - F.pr.nq);
        const float z = 1.0f - 2.0f * ua, r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
        float sp, cp;
        sincospif(2.0f * ub, &sp, &cp);
        y[0] = Sp[0] + Sp[3] * r * cp;
        y[1] = Sp[1] + Sp[3] * r * sp;
        y[2] = Sp[2] + Sp[3] * z;
    }
    const float nx = Q.nrm[3 * (size_t)s], ny = Q.nrm[3 * (size_t)s + 1], nz = Q.nrm[3 * (size_t)s + 2];
    const float ox = Q.pos[3 * (size_t)s] + F.offset * nx;
    const float oy = Q.pos[3 * (size_t)s + 1] + F.offset * ny;
    const float oz = Q.pos[3 * (size_t)s + 2] + F.offset * nz;
    const float ddx = y[0] - ox, ddy = y[1] - oy, ddz = y[2] - oz;
    const float dist = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
    float L = 0.0f, pl = 0.0f, wx = 0.0f, wy = 0.0f, wz = 1.0f;
    if (dist > 0.0f) {
        wx = ddx / dist;
        wy = ddy / dist;
        wz = ddz / dist;
        const float3 nl = prim_normal(F, prim, y[0], y[1], y[2]);
        pl = light_pdf(F, prim, dist, fabsf(nl.x * wx + nl.y * wy + nl.z * wz));
        const float cs = nx * wx + ny * wy + nz * wz;
        if (pl > 0.0f && cs > 0.0f) {
            const Hit h = frame_cast(F, ox, oy, oz, wx, wy, wz);
            if (h.prim == prim && fabsf(h.t - dist) <= 1e-3f * dist)
                L = (Q.alb[s] * kInvPi) * cs * F.emission[prim] / pl;
        }
    }
    store3(F.nee_dir, s, wx, wy, wz);
    F.nee_l[s] = L;
    F.nee_pl[s] = pl;
}

// Lambertian BSDF weight, closest hit (vertex k + 2), emission, roulette
__global__ void __launch_bounds__(256) k_shade(FrameView F, Queue Q, const float* __restrict__ dir,
                                               const float* __restrict__ pdf, Queue S, uint32_t* __restrict__ flags,
                                               int k) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= F.P) return;
    uint32_t flag = 0;
    if (s < F.counters[k]) {
        const uint32_t path = Q.path[s];
        const float nx = Q.nrm[3 * (size_t)s], ny = Q.nrm[3 * (size_t)s + 1], nz = Q.nrm[3 * (size_t)s + 2];
        const float dx = dir[3 * (size_t)s], dy = dir[3 * (size_t)s + 1], dz = dir[3 * (size_t)s + 2];
        const float p = pdf[s];
        const float cs = nx * dx + ny * dy + nz * dz;
        if (F.nee) {  // the light sample, weighed against the mixture by the power heuristic
            const float pl = F.nee_pl[s], pm = F.nee_pm[s];
            const float w = pl > 0.0f ? pl * pl / (pl * pl + pm * pm) : 0.0f;
            const size_t vc = (size_t)k * F.P + path;
            // per unit T(p_k): the continuation's roulette factor Q.T / T(p_k) applies
            const float tk = F.vT[vc];
            F.vNee[vc] = tk > 0.0f ? w * F.nee_l[s] * (Q.T[s] / tk) : 0.0f;
        }
        if (p > 0.0f && cs > 0.0f) {
            float T = Q.T[s] * (Q.alb[s] * kInvPi) * cs / p;
            const float ox = Q.pos[3 * (size_t)s] + F.offset * nx;
            const float oy = Q.pos[3 * (size_t)s + 1] + F.offset * ny;
            const float oz = Q.pos[3 * (size_t)s + 2] + F.offset * nz;
            const Hit h = frame_cast(F, ox, oy, oz, dx, dy, dz);
            if (h.prim != kNone) {
                const size_t v = (size_t)(k + 1) * F.P + path;
                const float hx = ox + h.t * dx, hy = oy + h.t * dy, hz = oz + h.t * dz;
                const float a = F.albedo[h.prim];
                F.vT[v] = T;
                const float Le = F.emission[h.prim];
                F.vLe[v] = Le;
                if (F.nee) {  // the mixture's sample of a light, weighed against light sampling
                    float w = 1.0f;
                    if (Le > 0.0f) {
                        const float3 nl = prim_normal(F, h.prim, hx, hy, hz);
                        const float pl = light_pdf(F, h.prim, h.t, fabsf(nl.x * dx + nl.y * dy + nl.z * dz));
                        w = p * p / (p * p + pl * pl);
                    }
                    F.vLw[v] = Le * w;
                    F.vNee[v] = 0.0f;
                }
                store3(F.vpos, v, hx, hy, hz);
                store3(F.vwo, v, -dx, -dy, -dz);
                F.nv[path] = (uint32_t)(k + 2);
                if (a > 0.0f && k + 1 < F.max_depth && roulette(F, path, k + 2, a, &T)) {
                    const float3 n = hit_normal(F.pr, h, ox, oy, oz, dx, dy, dz);
                    S.path[s] = path;
                    store3(S.pos, s, hx, hy, hz);
                    store3(S.nrm, s, n.x, n.y, n.z);
                    S.T[s] = T;
                    S.alb[s] = a;
                    flag = 1;
                }
            }
        }
    }
    flags[s] = flag;
}

// Eq. 5 for every vertex of every path, back to front: the suffix sum
// S_k = sum_{n >= k} T_n Le_n gives L_k = S_k / T_k; S_1 is the path estimate.
// The record array is compact in any order: each CTA reserves one run for all
// its records (one atomic per CTA), its warps take consecutive parts of it, and
// per vertex depth a warp's lanes that have that vertex write one contiguous
// piece, so every store instruction writes one run.
__global__ void __launch_bounds__(256) k_records(FrameView F, float* __restrict__ rec_pos,
                                                 float* __restrict__ rec_wout, float* __restrict__ rec_L,
                                                 uint32_t* __restrict__ rec_src) {
    __shared__ uint32_t s_warp[8], s_base;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    const int n = i < F.P ? (int)F.nv[i] : 0;
    int nmax = n, wtot = n;
    for (int o = 16; o > 0; o >>= 1) {
        nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        wtot += __shfl_xor_sync(0xffffffffu, wtot, o);
    }
    if (lane == 0) s_warp[warp] = (uint32_t)wtot;
    __syncthreads();
    if (threadIdx.x == 0) {  // the CTA's run, then each warp's part of it
        uint32_t tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const uint32_t c = s_warp[w];
            s_warp[w] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(&F.counters[WFPG_FRAME_MAX_DEPTH + 1], tot) : 0u;
    }
    __syncthreads();
    uint32_t base = s_base + s_warp[warp];
    // S: what the vertices after v contribute, as v sees them; Sv: v's own record (with NEE a
    // vertex's record holds its full emission, the vertex before it the MIS-weighted share)
    float S = 0.0f, Sv = 0.0f;
    for (int v = nmax - 1; v >= 0; --v) {
        const bool has = v < n;
        const uint32_t m = __ballot_sync(0xffffffffu, has);
        const uint32_t r = base + __popc(m & lt);
        base += __popc(m);
        if (!has) continue;
        const size_t e = (size_t)v * F.P + i;
        const float T = F.vT[e];
        Sv = S + T * (F.nee ? F.vLe[e] + F.vNee[e] : F.vLe[e]);
        S = F.nee ? S + T * (F.vLw[e] + F.vNee[e]) : Sv;
        rec_pos[3 * (size_t)r] = F.vpos[3 * e];
        rec_pos[3 * (size_t)r + 1] = F.vpos[3 * e + 1];
        rec_pos[3 * (size_t)r + 2] = F.vpos[3 * e + 2];
        rec_wout[3 * (size_t)r] = F.vwo[3 * e];
        rec_wout[3 * (size_t)r + 1] = F.vwo[3 * e + 1];
        rec_wout[3 * (size_t)r + 2] = F.vwo[3 * e + 2];
        rec_L[r] = Sv / T;
        rec_src[r] = (uint32_t)e;
    }
    if (i >= F.P) return;
    const double L = (double)Sv;
    F.img_sum[i] += L;
    F.img_sq[i] += L * L;
    F.img_wsum[i] += combine_weight(F.combine, *F.frames_run + 1ull) * L;
}

__global__ void k_frame_end(FrameView F) {
    unsigned long long g = 0;
    for (int k = 0; k < F.max_depth; ++k) g += F.counters[k];
    *F.guided += g;
    *F.wsum += combine_weight(F.combine, *F.frames_run + 1ull);
    *F.frames_run += 1ull;
    *F.frame_counter += 1u;
}

__global__ void __launch_bounds__(256) k_image(const double* __restrict__ sum, const double* __restrict__ sq,
                                               const double* __restrict__ wsum_px, const double* __restrict__ wsum,
                                               const unsigned long long* __restrict__ frames, uint32_t P,
                                               float* __restrict__ mean, float* __restrict__ var) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const double f = (double)*frames;
    const double m = f > 0 ? sum[i] / f : 0.0;
    if (mean) mean[i] = *wsum > 0.0 ? (float)(wsum_px[i] / *wsum) : 0.0f;
    if (var) var[i] = f > 1 ? (float)fmax(0.0, (sq[i] - f * m * m) / (f - 1.0)) : 0.0f;
}

// mean over pixels of the per-pixel variance (one block; for the autotuner)
__global__ void k_mean_var(const double* __restrict__ sum, const double* __restrict__ sq,
                           const unsigned long long* __restrict__ frames, uint32_t P, double* __restrict__ out) {
    __shared__ double red[256];
    const double f = (double)*frames;
    double acc = 0.0;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const double m = sum[i] / f;
        acc += fmax(0.0, (sq[i] - f * m * m) / (f - 1.0));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (double)P;
}

// The traced proposal's bins of one depth, split between the two field paths: all of them
// to the stream path (field tables, then the mixture sample) when they fit its tables, else
// all of them to the fused GuideRays launch.  The path that gets none does no work.
__global__ void k_split_bins(const uint32_t* __restrict__ n_bins, uint32_t cap, uint32_t* __restrict__ out) {
    const uint32_t nb = *n_bins;
    out[0] = nb <= cap ? nb : 0u;
    out[1] = nb <= cap ? 0u : nb;
}

}  // namespace wfpg

using namespace wfpg;

struct wfpg_frame {
    wfpg_svo* svo = nullptr;
    wfpg_scene scene{};
    const float* emission = nullptr;
    const float* albedo = nullptr;
    wfpg_camera cam{};
    wfpg_frame_params p{};
    int depth_cap = 0;  // max_depth the buffers were sized for
    uint32_t P = 0;
    uint32_t bin_cap = 0;
    std::vector<void*> allocs;
    Queue q[2]{}, stage{};
    uint32_t* flags = nullptr;
    uint32_t* offs = nullptr;
    float* dir = nullptr;
    float* pdf = nullptr;
    uint32_t* bin_of_ray = nullptr;
    uint32_t* ray_order = nullptr;
    uint32_t* bin_offset = nullptr;
    uint32_t* origin_ray = nullptr;
    uint32_t* n_bins = nullptr;  // [WFPG_FRAME_MAX_DEPTH + 1]
    void* bin_ws = nullptr;
    size_t bin_ws_bytes = 0;
    void* scan_ws = nullptr;
    size_t scan_ws_bytes = 0;
    void* guide_ws = nullptr;  // spill slots of the fused GuideRays launch (sized for N = 128)
    size_t guide_ws_bytes = 0;
    float* vT = nullptr;
    float* vLe = nullptr;
    float* vpos = nullptr;
    float* vwo = nullptr;
    uint32_t* nv = nullptr;
    float* rec_pos = nullptr;
    float* rec_wout = nullptr;
    float* rec_L = nullptr;
    uint32_t* rec_src = nullptr;
    double* img_sum = nullptr;
    double* img_sq = nullptr;
    double* img_wsum = nullptr;
    double* wsum = nullptr;
    unsigned long long frames_since_reset = 0;  // host-side count (PT first runs frame 1 unguided)
    uint32_t* counters = nullptr;  // [WFPG_FRAME_MAX_DEPTH + 2]
    uint32_t* fidx = nullptr;      // [WFPG_FRAME_MAX_DEPTH + 1]
    uint32_t* frame_counter = nullptr;
    unsigned long long* frames_run = nullptr;
    unsigned long long* guided = nullptr;
    double* scalar = nullptr;
    wfpg_mlp* mlp = nullptr;
    wfpg_learned_params lp{};
    float* probe_pos = nullptr;      // probe mode: the frame's copy of the probe points
    uint32_t n_lights = 0;           // emissive primitives (next-event estimation)
    uint32_t* light_prim = nullptr;
    float* light_cdf = nullptr;
    float* prim_pmf = nullptr;
    float* prim_area = nullptr;
    float* nee_dir = nullptr;
    float* nee_l = nullptr;
    float* nee_pl = nullptr;
    float* nee_pm = nullptr;
    float* vNee = nullptr;
    float* vLw = nullptr;
    uint32_t product_cap = 0;        // bins per depth the product tables hold
    int product_n = 0;               // grid side they are sized for
    float* prod_pdf = nullptr;       // [product_cap][N^2]
    float* prod_cr = nullptr;
    float* prod_cm = nullptr;        // [product_cap][N]
    float* prod_S = nullptr;         // [product_cap][64]
    uint32_t trace_cap = 0;          // bins per depth the traced proposal's tables hold (0: fused only)
    int trace_n = 0;                 // grid side they are sized for
    float* trace_pdf = nullptr;      // [trace_cap][N^2]
    float* trace_cr = nullptr;
    float* trace_cm = nullptr;       // [trace_cap][N]
    uint32_t* bin_split = nullptr;   // [WFPG_FRAME_MAX_DEPTH + 1][2]: bins of the stream path, of the fused launch
    uint32_t learned_cap = 0;        // bins per depth the learned tables hold
    float* tab_pdf = nullptr;        // [learned_cap][32 * 32]
    float* tab_cr = nullptr;
    float* tab_cm = nullptr;         // [learned_cap][32]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long graph_kernels = 0;
    ~wfpg_frame() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void* a : allocs) cudaFree(a);
    }
    template <typename T>
    bool alloc(T** out, size_t count) {
        void* ptr = nullptr;
        if (cudaMalloc(&ptr, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) return false;
        allocs.push_back(ptr);
        *out = static_cast<T*>(ptr);
        return true;
    }
    void release(void* ptr) {  // free one allocation of this frame (no graph may still use it)
        if (!ptr) return;
        auto it = std::find(allocs.begin(), allocs.end(), ptr);
        if (it != allocs.end()) allocs.erase(it);
        cudaFree(ptr);
    }
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    FrameView view() const {
        FrameView F;
        F.pr = prims_of(scene);
        F.emission = emission;
        F.albedo = albedo;
        F.P = P;
        F.W = cam.width;
        F.H = cam.height;
        const float th = tanf(cam.vfov_deg * 0.5f * 3.14159265358979f / 180.0f);
        const float aspect = (float)cam.width / (float)cam.height;
        const float* f = cam.forward;
        const float* u = cam.up;
        // image x grows along up x forward (+x for a camera looking along +z with +y up)
        const float r[3] = {u[1] * f[2] - u[2] * f[1], u[2] * f[0] - u[0] * f[2], u[0] * f[1] - u[1] * f[0]};
        for (int a = 0; a < 3; ++a) {
            F.eye[a] = cam.eye[a];
            F.fwd[a] = f[a];
            F.right[a] = r[a] * th * aspect;
            F.up[a] = u[a] * th;
        }
        F.probe_pos = probe_pos;
        F.probe_n = cam.probe_n;
        F.max_depth = p.max_depth;
        F.rr_depth = p.rr_depth;
        F.pseed = purpose(p.seed, kPathPurpose);
        F.offset = 1e-4f * scene.size;
        F.sv = svo_cast_view(svo);
        F.svo_cast = p.caster == 2 || (p.caster == 0 && scene.n_quads + scene.n_spheres + scene.n_tris > 64);
        F.vT = vT;
        F.vLe = vLe;
        F.vpos = vpos;
        F.vwo = vwo;
        F.nv = nv;
        F.img_sum = img_sum;
        F.img_sq = img_sq;
        F.img_wsum = img_wsum;
        F.wsum = wsum;
        F.combine = p.combine;
        F.nee = p.nee && n_lights > 0;
        F.n_lights = n_lights;
        F.light_prim = light_prim;
        F.light_cdf = light_cdf;
        F.prim_pmf = prim_pmf;
        F.prim_area = prim_area;
        F.nee_dir = nee_dir;
        F.nee_l = nee_l;
        F.nee_pl = nee_pl;
        F.nee_pm = nee_pm;
        F.vNee = vNee;
        F.vLw = vLw;
        F.counters = counters;
        F.fidx = fidx;
        F.frame_counter = frame_counter;
        F.frames_run = frames_run;
        F.guided = guided;
        return F;
    }
    // one frame's launches on st
    int enqueue(cudaStream_t st) {
        const FrameView F = view();
        const int T = 256;
        const uint32_t g = div_up(P, T);
        WFPG_LAUNCH(k_frame_begin, 1, 32, 0, st, F);
        WFPG_LAUNCH(k_camera, g, T, 0, st, F, stage, flags);
        for (int k = 0; k < p.max_depth; ++k) {
            Queue& Q = q[k & 1];
            {
                Arena ws{static_cast<char*>(scan_ws), scan_ws_bytes, 0, false};
                scan_exclusive(flags, offs, P, counters + k, ws, st);
            }
            WFPG_LAUNCH(k_compact, g, T, 0, st, F, stage, Q, flags, offs, k);
            const bool nee = F.nee != 0;
            if (nee) WFPG_LAUNCH(k_nee, g, T, 0, st, F, Q, k);
            wfpg_bin_params bp{};
            bp.mode = WFPG_BIN_PARTITION_S;
            bp.l_min = p.l_min;
            bp.c_ray = p.c_ray;
            bp.seed = p.seed;
            bp.n_dev = counters + k;
            int rc = bin_rays_impl(svo, Q.pos, Q.nrm, P, &bp, nullptr, bin_of_ray, ray_order, bin_offset, origin_ray,
                                   bin_cap, n_bins + k, bin_ws, bin_ws_bytes, st, fidx + k);
            if (rc != WFPG_OK) return rc;
            if (p.proposal == 2) {  // product guiding (Sec. 3.6): field tables, block sums, two-stage sample
                wfpg_guide_params gp = p.guide;
                gp.seed = p.seed;
                if (p.decay) gp.N = std::max(8, p.guide.N >> k);
                rc = guide_build_impl(svo, Q.pos, origin_ray, n_bins + k, product_cap, &gp, prod_pdf, prod_cr,
                                      prod_cm, st, fidx + k);
                if (rc == WFPG_OK) rc = product_sums_impl(prod_pdf, gp.N, product_cap, n_bins + k, prod_S, st);
                if (rc == WFPG_OK)
                    rc = product_sample_impl(prod_pdf, prod_S, gp.N, product_cap, n_bins + k, bin_of_ray, Q.nrm,
                                             Q.u, P, counters + k, p.alpha, dir, pdf, nullptr, st);
                if (rc == WFPG_OK && nee)
                    rc = product_eval_impl(prod_pdf, prod_S, gp.N, product_cap, n_bins + k, bin_of_ray, Q.nrm, nee_dir,
                                           P, p.alpha, nee_pm, st, counters + k);
            } else if (p.proposal == 1) {  // learned: MLP tables for the bins' origins, then the mixture
                if (!mlp) return WFPG_ERR_INVALID_ARG;
                rc = guide_learned_build_pdf(mlp, Q.pos, Q.nrm, origin_ray, n_bins + k, learned_cap, &lp, tab_pdf,
                                             tab_cr, tab_cm, st);
                if (rc != WFPG_OK) return rc;
                rc = sample_mix_impl(tab_pdf, tab_cr, tab_cm, 32, learned_cap, n_bins + k, bin_of_ray, Q.nrm, Q.u, P,
                                     counters + k, p.alpha, dir, pdf, st);
                if (rc == WFPG_OK && nee)
                    rc = mix_eval_impl(tab_pdf, 32, learned_cap, n_bins + k, bin_of_ray, Q.nrm, nee_dir, P,
                                       counters + k, p.alpha, nee_pm, st);
            } else {
                wfpg_guide_params gp = p.guide;
                gp.seed = p.seed;
                if (p.decay) gp.N = std::max(8, p.guide.N >> k);
                const uint32_t* fused_bins = n_bins + k;
                if (trace_cap > 0) {
                    // the stream field kernel into tables, then the mixture sample (bit-identical
                    // to the fused launch); the fused launch takes over when the bins overflow
                    uint32_t* split = bin_split + 2 * k;
                    WFPG_LAUNCH(k_split_bins, 1, 1, 0, st, n_bins + k, trace_cap, split);
                    rc = guide_build_impl(svo, Q.pos, origin_ray, split, trace_cap, &gp, trace_pdf, trace_cr,
                                          trace_cm, st, fidx + k);
                    if (rc == WFPG_OK)
                        rc = sample_mix_impl(trace_pdf, trace_cr, trace_cm, gp.N, trace_cap, split, bin_of_ray, Q.nrm,
                                             Q.u, P, counters + k, p.alpha, dir, pdf, st);
                    if (rc == WFPG_OK && nee)
                        rc = mix_eval_impl(trace_pdf, gp.N, trace_cap, split, bin_of_ray, Q.nrm, nee_dir, P,
                                           counters + k, p.alpha, nee_pm, st);
                    fused_bins = split + 1;
                }
                if (rc == WFPG_OK)
                    rc = guide_fused_impl(svo, Q.pos, Q.nrm, origin_ray, fused_bins, bin_cap, ray_order, bin_offset,
                                          Q.u, p.alpha, &gp, dir, pdf, P, guide_ws, guide_ws_bytes, st, fidx + k,
                                          nee ? nee_dir : nullptr, nee ? nee_pm : nullptr);
            }
            if (rc != WFPG_OK) return rc;
            WFPG_LAUNCH(k_shade, g, T, 0, st, F, Q, dir, pdf, stage, flags, k);
        }
        WFPG_LAUNCH(k_records, g, T, 0, st, F, rec_pos, rec_wout, rec_L, rec_src);
        if (p.update) {
            const int rc = accumulate(svo, rec_pos, rec_wout, rec_L, (uint32_t)((size_t)(p.max_depth + 1) * P), st,
                                      counters + WFPG_FRAME_MAX_DEPTH + 1);
            if (rc != WFPG_OK) return rc;
        }
        WFPG_LAUNCH(k_frame_end, 1, 1, 0, st, F);
        return launch_status();
    }
    // tables for the traced proposal's stream path, allocated outside any capture (kept for the
    // frame's lifetime): only with the SVO's flat index (top index and occupancy bitmaps), at most
    // 64M floats per table (65,536 bins at N = 32, 16,384 at 64, 4,096 at 128)
    bool ensure_trace_tables() {
        const bool flat = svo->top_levels > 0 && (svo->top_levels - 1 == svo->D || svo->occ != nullptr);
        if (p.proposal != 0 || !flat || p.guide.parts != 0) return true;
        const size_t NN = (size_t)p.guide.N * p.guide.N;
        const uint32_t cap = (uint32_t)std::min<size_t>({(size_t)bin_cap, 65536u, ((size_t)64 << 20) / NN});
        if (cap <= trace_cap && p.guide.N <= trace_n) return true;
        release(trace_pdf);
        release(trace_cr);
        release(trace_cm);
        trace_pdf = trace_cr = trace_cm = nullptr;
        trace_cap = 0;
        trace_n = 0;
        if (!alloc(&trace_pdf, cap * NN) || !alloc(&trace_cr, cap * NN) || !alloc(&trace_cm, (size_t)cap * p.guide.N)) {
            cudaGetLastError();
            return false;
        }
        trace_cap = cap;
        trace_n = p.guide.N;
        return true;
    }
    // tables for the product proposal, allocated outside any capture (kept for the frame's lifetime)
    bool ensure_product_tables() {
        if (p.proposal != 2) return true;
        const uint32_t cap = std::min<uint32_t>(bin_cap, 65536u);
        if (cap <= product_cap && p.guide.N <= product_n) return true;
        const size_t NN = (size_t)p.guide.N * p.guide.N;
        if (!alloc(&prod_pdf, cap * NN) || !alloc(&prod_cr, cap * NN) || !alloc(&prod_cm, (size_t)cap * p.guide.N) ||
            !alloc(&prod_S, (size_t)cap * 64)) {
            cudaGetLastError();
            return false;
        }
        product_cap = cap;
        product_n = p.guide.N;
        return true;
    }
    int capture(cudaStream_t st) {
        drop_graph();
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return WFPG_ERR_CUDA;
        const unsigned long long before = wfpg_kernel_launches();
        int rc = WFPG_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = WFPG_ERR_CUDA;
        if (rc == WFPG_OK) {
            rc = enqueue(cs);
            const cudaError_t e = cudaStreamEndCapture(cs, &graph);
            if (rc == WFPG_OK && e != cudaSuccess) rc = WFPG_ERR_CUDA;
        }
        graph_kernels = wfpg_kernel_launches() - before;
        note_launches(-(long long)graph_kernels);  // captured launches run only when replayed
        if (rc == WFPG_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = WFPG_ERR_CUDA;
        cudaStreamDestroy(cs);
        if (rc != WFPG_OK) drop_graph();
        (void)st;
        return rc;
    }
};

static int ffail(int code, const char* msg) { return set_last_error(code, msg); }

static bool valid_grid_n(int N) { return N == 8 || N == 16 || N == 32 || N == 64 || N == 128; }

static int check_params(const wfpg_frame_params* p, int depth_cap) {
    if (!p) return ffail(WFPG_ERR_INVALID_ARG, "frame: null params");
    if (p->max_depth < 1 || p->max_depth > WFPG_FRAME_MAX_DEPTH || (depth_cap && p->max_depth > depth_cap))
        return ffail(WFPG_ERR_INVALID_ARG, "frame: max_depth out of range");
    if (!(p->alpha >= 0.0f && p->alpha <= 1.0f)) return ffail(WFPG_ERR_INVALID_ARG, "frame: alpha must be in [0, 1]");
    if (!valid_grid_n(p->guide.N)) return ffail(WFPG_ERR_INVALID_ARG, "frame: N must be 8, 16, 32, 64 or 128");
    if (!(p->guide.eps >= 0.0f)) return ffail(WFPG_ERR_INVALID_ARG, "frame: eps must be >= 0");
    if (p->guide.block != 0 && p->guide.block != 64 && p->guide.block != 128 && p->guide.block != 256)
        return ffail(WFPG_ERR_INVALID_ARG, "frame: block must be 0, 64, 128 or 256");
    if (p->c_ray == 0) return ffail(WFPG_ERR_INVALID_ARG, "frame: c_ray must be >= 1");
    if (p->guide.split != 0 && p->guide.split != 0xFFFFFFFFu && p->guide.split < 2048)
        return ffail(WFPG_ERR_INVALID_ARG, "frame: guide.split must be 0, >= 2048 or 0xFFFFFFFF");
    if (p->caster < 0 || p->caster > 2) return ffail(WFPG_ERR_INVALID_ARG, "frame: caster must be 0, 1 or 2");
    if (p->proposal < 0 || p->proposal > 2) return ffail(WFPG_ERR_INVALID_ARG, "frame: proposal must be 0, 1 or 2");
    if (p->proposal == 1 && p->guide.N != 32)
        return ffail(WFPG_ERR_INVALID_ARG, "frame: the learned proposal has N = 32");
    if (p->combine < 0 || p->combine > 5) return ffail(WFPG_ERR_INVALID_ARG, "frame: combine must be 0 .. 5");
    if (p->nee != 0 && p->nee != 1) return ffail(WFPG_ERR_INVALID_ARG, "frame: nee must be 0 or 1");
    return WFPG_OK;
}

extern "C" {

int frame_create(wfpg_svo* svo, const wfpg_scene* scene, const float* emission, const float* albedo,
                 const wfpg_camera* cam, const wfpg_frame_params* p, wfpg_frame** out, void* stream) {
    if (!svo || !scene || !emission || !albedo || !cam || !out)
        return ffail(WFPG_ERR_INVALID_ARG, "frame_create: null argument");
    *out = nullptr;
    // record slots (max_depth + 1) x W x H are addressed with 32-bit indices
    if (cam->width == 0 || cam->height == 0 ||
        (uint64_t)cam->width * cam->height * (uint64_t)(WFPG_FRAME_MAX_DEPTH + 1) > 0xFFFFFFFFull)
        return ffail(WFPG_ERR_INVALID_ARG, "frame_create: image size out of range");
    if (!cam->probe_pos && !(cam->vfov_deg > 0.0f && cam->vfov_deg < 180.0f))
        return ffail(WFPG_ERR_INVALID_ARG, "frame_create: vfov_deg must be in (0, 180)");
    if (cam->probe_pos && (cam->probe_n == 0 || cam->probe_n > 1024 || cam->width != cam->probe_n * cam->probe_n))
        return ffail(WFPG_ERR_INVALID_ARG, "frame_create: probe mode needs 1 <= probe_n <= 1024 and width = probe_n^2");
    if (const int rc = check_params(p, 0)) return rc;
    auto* f = new wfpg_frame();
    f->svo = svo;
    f->scene = *scene;
    f->emission = emission;
    f->albedo = albedo;
    f->cam = *cam;
    f->p = *p;
    f->depth_cap = p->max_depth;
    const uint32_t P = cam->width * cam->height;
    f->P = P;
    f->bin_cap = std::max<uint32_t>(1, std::min<uint32_t>(P, svo->n_nodes));
    const size_t V = (size_t)(p->max_depth + 1) * P;
    bool ok = true;
    for (int j = 0; j < 3; ++j) {
        Queue& Q = j < 2 ? f->q[j] : f->stage;
        ok = ok && f->alloc(&Q.path, P) && f->alloc(&Q.pos, 3 * (size_t)P) && f->alloc(&Q.nrm, 3 * (size_t)P) &&
             f->alloc(&Q.T, P) && f->alloc(&Q.alb, P);
        if (j < 2) ok = ok && f->alloc(&Q.u, 3 * (size_t)P);
    }
    f->bin_ws_bytes = bin_workspace_bytes(svo, P, WFPG_BIN_PARTITION_S, 0);
    f->scan_ws_bytes = scan_workspace_bytes(P) + 1024;
    f->guide_ws_bytes = guide_fused_workspace_bytes(128, P, 0);
    ok = ok && f->alloc(&f->flags, P) && f->alloc(&f->offs, P) && f->alloc(&f->dir, 3 * (size_t)P) &&
         f->alloc(&f->pdf, P) && f->alloc(&f->bin_of_ray, P) && f->alloc(&f->ray_order, P) &&
         f->alloc(&f->bin_offset, (size_t)f->bin_cap + 1) && f->alloc(&f->origin_ray, f->bin_cap) &&
         f->alloc(&f->n_bins, WFPG_FRAME_MAX_DEPTH + 1) &&
         f->alloc(reinterpret_cast<char**>(&f->bin_ws), f->bin_ws_bytes) &&
         f->alloc(reinterpret_cast<char**>(&f->scan_ws), f->scan_ws_bytes) &&
         f->alloc(reinterpret_cast<char**>(&f->guide_ws), f->guide_ws_bytes) && f->alloc(&f->vT, V) &&
         f->alloc(&f->vLe, V) && f->alloc(&f->vpos, 3 * V) && f->alloc(&f->vwo, 3 * V) && f->alloc(&f->nv, P) &&
         f->alloc(&f->rec_pos, 3 * V) && f->alloc(&f->rec_wout, 3 * V) && f->alloc(&f->rec_L, V) &&
         f->alloc(&f->rec_src, V) && f->alloc(&f->img_sum, P) && f->alloc(&f->img_sq, P) &&
         f->alloc(&f->img_wsum, P) && f->alloc(&f->wsum, 1) &&
         f->alloc(&f->counters, WFPG_FRAME_MAX_DEPTH + 2) && f->alloc(&f->fidx, WFPG_FRAME_MAX_DEPTH + 1) &&
         f->alloc(&f->frame_counter, 1) && f->alloc(&f->frames_run, 1) && f->alloc(&f->guided, 1) &&
         f->alloc(&f->scalar, 1) && f->alloc(&f->bin_split, 2 * (WFPG_FRAME_MAX_DEPTH + 1));
    if (!ok) {
        delete f;
        cudaGetLastError();
        return ffail(WFPG_ERR_OOM, "frame_create: device allocation failed");
    }
    if (!f->ensure_product_tables() || !f->ensure_trace_tables()) {
        delete f;
        return ffail(WFPG_ERR_OOM, "frame_create: device allocation of the guiding tables failed");
    }
    if (cam->probe_pos) {
        if (!f->alloc(&f->probe_pos, 3 * (size_t)cam->height) ||
            cudaMemcpy(f->probe_pos, cam->probe_pos, 12 * (size_t)cam->height, cudaMemcpyDeviceToDevice) != cudaSuccess) {
            delete f;
            cudaGetLastError();
            return ffail(WFPG_ERR_INVALID_ARG, "frame_create: probe points could not be copied");
        }
    }
    // next-event estimation: the emissive primitives, chosen in proportion to emitted power
    {
        const uint32_t nq = scene->n_quads, ns = scene->n_spheres, nt = scene->n_tris, np = nq + ns + nt;
        std::vector<float> hq(8 * (size_t)nq), hs(4 * (size_t)ns), ht(9 * (size_t)nt), he(np);
        bool okc = (nq == 0 || cudaMemcpy(hq.data(), scene->quads, 4 * hq.size(), cudaMemcpyDeviceToHost) == cudaSuccess) &&
                   (ns == 0 || cudaMemcpy(hs.data(), scene->spheres, 4 * hs.size(), cudaMemcpyDeviceToHost) == cudaSuccess) &&
                   (nt == 0 || cudaMemcpy(ht.data(), scene->tris, 4 * ht.size(), cudaMemcpyDeviceToHost) == cudaSuccess) &&
                   (np == 0 || cudaMemcpy(he.data(), emission, 4 * he.size(), cudaMemcpyDeviceToHost) == cudaSuccess);
        std::vector<float> area(np, 0.0f), pmf(np, 0.0f);
        std::vector<uint32_t> lp;
        std::vector<double> power;
        double total = 0.0;
        for (uint32_t k = 0; okc && k < np; ++k) {
            if (k < nq) {
                area[k] = (hq[8 * k + 3] - hq[8 * k + 2]) * (hq[8 * k + 5] - hq[8 * k + 4]);
            } else if (k < nq + ns) {
                area[k] = 12.566370614359172f * hs[4 * (k - nq) + 3] * hs[4 * (k - nq) + 3];
            } else {
                const float* T = ht.data() + 9 * (size_t)(k - nq - ns);
                const double e1[3] = {(double)T[3] - T[0], (double)T[4] - T[1], (double)T[5] - T[2]};
                const double e2[3] = {(double)T[6] - T[0], (double)T[7] - T[1], (double)T[8] - T[2]};
                const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                     e1[0] * e2[1] - e1[1] * e2[0]};
                area[k] = (float)(0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]));
            }
            if (he[k] > 0.0f && area[k] > 0.0f) {
                lp.push_back(k);
                power.push_back((double)he[k] * area[k]);
                total += power.back();
            }
        }
        std::vector<float> cdf(lp.size());
        double acc = 0.0;
        for (size_t j = 0; j < lp.size(); ++j) {
            acc += power[j];
            cdf[j] = j + 1 == lp.size() ? 1.0f : (float)(acc / total);
            pmf[lp[j]] = (float)(power[j] / total);
        }
        f->n_lights = (uint32_t)lp.size();
        const size_t V2 = (size_t)(p->max_depth + 1) * P;
        okc = okc && f->alloc(&f->light_prim, std::max<size_t>(1, lp.size())) &&
              f->alloc(&f->light_cdf, std::max<size_t>(1, lp.size())) && f->alloc(&f->prim_pmf, std::max<uint32_t>(1, np)) &&
              f->alloc(&f->prim_area, std::max<uint32_t>(1, np)) && f->alloc(&f->nee_dir, 3 * (size_t)P) &&
              f->alloc(&f->nee_l, P) && f->alloc(&f->nee_pl, P) && f->alloc(&f->nee_pm, P) && f->alloc(&f->vNee, V2) &&
              f->alloc(&f->vLw, V2);
        okc = okc && (lp.empty() || (cudaMemcpy(f->light_prim, lp.data(), 4 * lp.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                                     cudaMemcpy(f->light_cdf, cdf.data(), 4 * cdf.size(), cudaMemcpyHostToDevice) == cudaSuccess)) &&
              (np == 0 || (cudaMemcpy(f->prim_pmf, pmf.data(), 4 * (size_t)np, cudaMemcpyHostToDevice) == cudaSuccess &&
                           cudaMemcpy(f->prim_area, area.data(), 4 * (size_t)np, cudaMemcpyHostToDevice) == cudaSuccess));
        if (!okc) {
            delete f;
            cudaGetLastError();
            return ffail(WFPG_ERR_OOM, "frame_create: light table setup failed");
        }
    }
    auto st = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(f->counters, 0, 4 * (WFPG_FRAME_MAX_DEPTH + 2), st);
    cudaMemsetAsync(f->n_bins, 0, 4 * (WFPG_FRAME_MAX_DEPTH + 1), st);
    cudaMemsetAsync(f->nv, 0, 4 * (size_t)P, st);
    cudaMemsetAsync(f->img_sum, 0, 8 * (size_t)P, st);
    cudaMemsetAsync(f->img_sq, 0, 8 * (size_t)P, st);
    cudaMemsetAsync(f->img_wsum, 0, 8 * (size_t)P, st);
    cudaMemsetAsync(f->wsum, 0, 8, st);
    cudaMemsetAsync(f->frame_counter, 0, 4, st);
    cudaMemsetAsync(f->frames_run, 0, 8, st);
    cudaMemsetAsync(f->guided, 0, 8, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        delete f;
        return ffail(WFPG_ERR_CUDA, "frame_create: initialisation failed");
    }
    *out = f;
    return WFPG_OK;
}

int frame_destroy(wfpg_frame* f) {
    if (f) {
        cudaDeviceSynchronize();
        delete f;
    }
    return WFPG_OK;
}

int frame_run(wfpg_frame* f, uint32_t n_frames, int use_graph, void* stream) {
    if (!f) return ffail(WFPG_ERR_INVALID_ARG, "frame_run: null frame");
    if (f->p.proposal == 1 && !f->mlp) return ffail(WFPG_ERR_INVALID_ARG, "frame_run: learned proposal without MLP");
    auto st = static_cast<cudaStream_t>(stream);
    if (use_graph && !f->exec) {
        const int rc = f->capture(st);
        if (rc != WFPG_OK) return ffail(rc, "frame_run: graph capture failed");
    }
    for (uint32_t i = 0; i < n_frames; ++i) {
        if (f->p.combine == 5 && f->frames_since_reset == 0) {  // PT first: the first frame unguided
            const float alpha = f->p.alpha;
            f->p.alpha = 0.0f;
            const int rc = f->enqueue(st);
            f->p.alpha = alpha;
            ++f->frames_since_reset;
            if (rc != WFPG_OK) return ffail(rc, "frame_run: launch failed");
            continue;
        }
        ++f->frames_since_reset;
        if (use_graph) {
            if (cudaGraphLaunch(f->exec, st) != cudaSuccess) return ffail(WFPG_ERR_CUDA, "frame_run: graph launch");
            note_launches((long long)f->graph_kernels);
        } else {
            const int rc = f->enqueue(st);
            if (rc != WFPG_OK) return ffail(rc, "frame_run: launch failed");
        }
    }
    return WFPG_OK;
}

int frame_set_params(wfpg_frame* f, const wfpg_frame_params* p) {
    if (!f) return ffail(WFPG_ERR_INVALID_ARG, "frame_set_params: null frame");
    if (const int rc = check_params(p, f->depth_cap)) return rc;
    f->drop_graph();
    const wfpg_frame_params old = f->p;
    f->p = *p;
    if (!f->ensure_product_tables() || !f->ensure_trace_tables()) {
        f->p = old;
        return ffail(WFPG_ERR_OOM, "frame_set_params: device allocation of the guiding tables failed");
    }
    return WFPG_OK;
}

int frame_set_mlp(wfpg_frame* f, wfpg_mlp* mlp, const wfpg_learned_params* lp) {
    if (!f || (mlp && !lp)) return ffail(WFPG_ERR_INVALID_ARG, "frame_set_mlp: null argument");
    f->drop_graph();
    f->mlp = mlp;
    if (!mlp) return WFPG_OK;
    f->lp = *lp;
    const uint32_t cap = std::min(f->bin_cap, mlp_max_batch(mlp));
    if (cap > f->learned_cap) {  // grow the tables (kept for the frame's lifetime)
        if (!f->alloc(&f->tab_pdf, (size_t)cap * 1024) || !f->alloc(&f->tab_cr, (size_t)cap * 1024) ||
            !f->alloc(&f->tab_cm, (size_t)cap * 32)) {
            cudaGetLastError();
            f->mlp = nullptr;
            return ffail(WFPG_ERR_OOM, "frame_set_mlp: device allocation failed");
        }
    }
    f->learned_cap = cap;
    return WFPG_OK;
}

int frame_get_params(const wfpg_frame* f, wfpg_frame_params* p) {
    if (!f || !p) return ffail(WFPG_ERR_INVALID_ARG, "frame_get_params: null argument");
    *p = f->p;
    return WFPG_OK;
}

int frame_reset_image(wfpg_frame* f, void* stream) {
    if (!f) return ffail(WFPG_ERR_INVALID_ARG, "frame_reset_image: null frame");
    auto st = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(f->img_sum, 0, 8 * (size_t)f->P, st);
    cudaMemsetAsync(f->img_sq, 0, 8 * (size_t)f->P, st);
    cudaMemsetAsync(f->img_wsum, 0, 8 * (size_t)f->P, st);
    cudaMemsetAsync(f->wsum, 0, 8, st);
    f->frames_since_reset = 0;
    cudaMemsetAsync(f->frames_run, 0, 8, st);
    cudaMemsetAsync(f->guided, 0, 8, st);
    return cudaGetLastError() == cudaSuccess ? WFPG_OK : ffail(WFPG_ERR_CUDA, "frame_reset_image");
}

int frame_image(wfpg_frame* f, float* mean, float* var, void* stream) {
    if (!f) return ffail(WFPG_ERR_INVALID_ARG, "frame_image: null frame");
    WFPG_LAUNCH(k_image, div_up(f->P, 256), 256, 0, static_cast<cudaStream_t>(stream), f->img_sum, f->img_sq,
                f->img_wsum, f->wsum, f->frames_run, f->P, mean, var);
    return cudaGetLastError() == cudaSuccess ? WFPG_OK : ffail(WFPG_ERR_CUDA, "frame_image");
}

int frame_stats(wfpg_frame* f, wfpg_frame_stats* out, void* stream) {
    if (!f || !out) return ffail(WFPG_ERR_INVALID_ARG, "frame_stats: null argument");
    auto st = static_cast<cudaStream_t>(stream);
    uint32_t c[WFPG_FRAME_MAX_DEPTH + 2], nb[WFPG_FRAME_MAX_DEPTH + 1];
    unsigned long long fr = 0, g = 0;
    uint32_t status = 0;
    cudaMemcpyAsync(c, f->counters, sizeof c, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(nb, f->n_bins, sizeof nb, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&fr, f->frames_run, 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&g, f->guided, 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&status, f->svo->status, 4, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return ffail(WFPG_ERR_CUDA, "frame_stats: copy failed");
    std::memset(out, 0, sizeof *out);
    out->frames = fr;
    for (int k = 0; k < f->p.max_depth; ++k) {
        out->paths[k] = c[k];
        out->bins[k] = nb[k];
    }
    out->records = c[WFPG_FRAME_MAX_DEPTH + 1];
    out->guided_samples = g;
    out->status = status;
    out->kernels_per_frame = f->graph_kernels;
    return WFPG_OK;
}

int frame_autotune(wfpg_frame* f, const int* N_candidates, int n_N, uint32_t frames, wfpg_frame_params* chosen,
                   float* ms_per_frame, void* stream) {
    if (!f || !N_candidates || n_N < 1 || frames < 2)
        return ffail(WFPG_ERR_INVALID_ARG, "frame_autotune: need candidates and frames >= 2");
    for (int i = 0; i < n_N; ++i)
        if (!valid_grid_n(N_candidates[i])) return ffail(WFPG_ERR_INVALID_ARG, "frame_autotune: bad N candidate");
    auto st = static_cast<cudaStream_t>(stream);
    const wfpg_frame_params base = f->p;
    static const int kTiles[6][2] = {{64, 1}, {64, -1}, {128, 1}, {128, -1}, {256, 1}, {256, -1}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_fom = -1.0;
    wfpg_frame_params best = base;
    float best_ms = 0.0f;
    int rc = WFPG_OK;
    for (int i = 0; i < n_N && rc == WFPG_OK; ++i) {
        wfpg_frame_params t = base;
        t.guide.N = N_candidates[i];
        float tile_ms = -1.0f;
        wfpg_frame_params tile_best = t;
        for (const auto& tile : kTiles) {
            t.guide.block = tile[0];
            t.guide.stage = tile[1];
            f->p = t;
            f->drop_graph();
            if (f->capture(st) != WFPG_OK) {  // this tile does not fit (shared memory): skip it
                cudaGetLastError();
                continue;
            }
            // the best of three runs of three frames each (after one warm frame): tiles within a
            // few percent of each other are told apart only above the run-to-run noise
            cudaGraphLaunch(f->exec, st);
            float ms = -1.0f;
            for (int rep = 0; rep < 3 && rc == WFPG_OK; ++rep) {
                cudaEventRecord(e0, st);
                for (int k = 0; k < 3; ++k) cudaGraphLaunch(f->exec, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = WFPG_ERR_CUDA;
                    break;
                }
                float m = 0.0f;
                cudaEventElapsedTime(&m, e0, e1);
                m /= 3.0f;
                if (ms < 0.0f || m < ms) ms = m;
            }
            note_launches(10ll * (long long)f->graph_kernels);
            if (rc != WFPG_OK) break;
            if (tile_ms < 0.0f || ms < tile_ms) {
                tile_ms = ms;
                tile_best = t;
            }
        }
        if (rc != WFPG_OK || tile_ms < 0.0f) continue;
        f->p = tile_best;
        f->drop_graph();
        if (f->capture(st) != WFPG_OK) continue;
        frame_reset_image(f, st);
        for (uint32_t k = 0; k < frames; ++k) cudaGraphLaunch(f->exec, st);
        note_launches((long long)frames * (long long)f->graph_kernels);
        WFPG_LAUNCH(k_mean_var, 1, 256, 0, st, f->img_sum, f->img_sq, f->frames_run, f->P, f->scalar);
        double mv = 0.0;
        cudaMemcpyAsync(&mv, f->scalar, 8, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = WFPG_ERR_CUDA;
            break;
        }
        const double fom = mv * (double)tile_ms;
        if (best_fom < 0.0 || fom < best_fom) {
            best_fom = fom;
            best = tile_best;
            best_ms = tile_ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != WFPG_OK) {
        f->p = base;
        f->drop_graph();
        return ffail(rc, "frame_autotune: CUDA error");
    }
    if (best_fom < 0.0) {
        f->p = base;
        f->drop_graph();
        return ffail(WFPG_ERR_INVALID_ARG, "frame_autotune: no candidate fits");
    }
    f->p = best;
    f->drop_graph();
    frame_reset_image(f, st);
    if (chosen) *chosen = best;
    if (ms_per_frame) *ms_per_frame = best_ms;
    return cudaStreamSynchronize(st) == cudaSuccess ? WFPG_OK : ffail(WFPG_ERR_CUDA, "frame_autotune");
}

int frame_export(const wfpg_frame* f, int what, void* dst, size_t bytes, void* stream) {
    if (!f || !dst) return ffail(WFPG_ERR_INVALID_ARG, "frame_export: null argument");
    const size_t P = f->P, V = (size_t)(f->depth_cap + 1) * P;
    const int last = (f->p.max_depth - 1) & 1;
    const void* src = nullptr;
    size_t n = 0;
    switch (what) {
        case WFPG_FRAME_BUF_VT: src = f->vT; n = 4 * V; break;
        case WFPG_FRAME_BUF_VLE: src = f->vLe; n = 4 * V; break;
        case WFPG_FRAME_BUF_VPOS: src = f->vpos; n = 12 * V; break;
        case WFPG_FRAME_BUF_VWO: src = f->vwo; n = 12 * V; break;
        case WFPG_FRAME_BUF_NV: src = f->nv; n = 4 * P; break;
        case WFPG_FRAME_BUF_REC_POS: src = f->rec_pos; n = 12 * V; break;
        case WFPG_FRAME_BUF_REC_WOUT: src = f->rec_wout; n = 12 * V; break;
        case WFPG_FRAME_BUF_REC_L: src = f->rec_L; n = 4 * V; break;
        case WFPG_FRAME_BUF_REC_SRC: src = f->rec_src; n = 4 * V; break;
        case WFPG_FRAME_BUF_Q_POS: src = f->q[last].pos; n = 12 * P; break;
        case WFPG_FRAME_BUF_Q_NRM: src = f->q[last].nrm; n = 12 * P; break;
        case WFPG_FRAME_BUF_Q_U: src = f->q[last].u; n = 12 * P; break;
        case WFPG_FRAME_BUF_Q_DIR: src = f->dir; n = 12 * P; break;
        case WFPG_FRAME_BUF_Q_PDF: src = f->pdf; n = 4 * P; break;
        case WFPG_FRAME_BUF_Q_PATH: src = f->q[last].path; n = 4 * P; break;
        case WFPG_FRAME_BUF_VNEE: src = f->vNee; n = 4 * V; break;
        case WFPG_FRAME_BUF_NEE_DIR: src = f->nee_dir; n = 12 * P; break;
        case WFPG_FRAME_BUF_NEE_PL: src = f->nee_pl; n = 4 * P; break;
        case WFPG_FRAME_BUF_NEE_PM: src = f->nee_pm; n = 4 * P; break;
        case WFPG_FRAME_BUF_NEE_L: src = f->nee_l; n = 4 * P; break;
        case WFPG_FRAME_BUF_VLW: src = f->vLw; n = 4 * V; break;
        default: return ffail(WFPG_ERR_INVALID_ARG, "frame_export: unknown buffer");
    }
    if (bytes != n) return ffail(WFPG_ERR_INVALID_ARG, "frame_export: size mismatch");
    if (cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return ffail(WFPG_ERR_CUDA, "frame_export: copy failed");
    return WFPG_OK;
}

}  // extern "C"
