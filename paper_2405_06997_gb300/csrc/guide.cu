// GuideRays (Alg. 3): per-bin cone-traced radiance field (Sec. 3.3, Eq. 6),
// epsilon floor, blur, warp-scan CDFs and PDF (Sec. 3.5), then inverse-CDF
// sampling and PDF evaluation for MIS.
//
// One CTA owns one bin at a time (persistent over bins): its threads march
// the N x N cell rays through the SVO -- the top levels staged in shared
// memory, deeper nodes read as 8-byte records through the read-only path --
// the field, its blur and its scans stay in shared memory, and only the
// finished pdf / cdf_row / cdf_marg rows go to global memory.
//
// The SVO march returns exactly the leaf that a leaf-by-leaf 3D DDA returns:
// every boundary time is evaluated afresh as (k - g) / (d * 2^D / S) for an
// integer boundary k; when the walk sits in an empty block it jumps to the
// block's exit crossing (the smallest face time, ties x < y < z) and sets the
// other coordinates to the cells a leaf-by-leaf walk would have reached by
// that crossing (crossings earlier in (time, axis) order).
#include "common.cuh"
#include "svo.cuh"

namespace wfpg {

constexpr float kOneMinus = 0x1.fffffep-1f;
constexpr int kGuideThreads = 256;
constexpr int kSmemTopLevels = 3;  // levels 0..3 of the SVO (<= 585 nodes) live in shared memory

struct TraceArgs {
    const Node* node;
    const float4* normal;
    const float2* value;
    int D;
    float lo[3];
    float scale;
    float S;
    float t_skip;
    float omega;
    int cos_weight;
    uint32_t smem_nodes;
};

struct GuideArgs {
    int N;
    float eps;
    int jitter;
    int blur;
    uint64_t seed;
    uint32_t frame;
};

__device__ __forceinline__ Node load_node(const TraceArgs& T, const Node* s_nodes, uint32_t id) {
    if (id < T.smem_nodes) return s_nodes[id];
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(T.node) + id);
    Node n;
    n.first_child = v.x;
    n.mask = v.y;
    return n;
}

// crossing into cell j along axis b (moving in direction st) happens at the
// boundary j (st > 0) or j + 1 (st < 0); "before (tx, a)" in (time, axis) order
__device__ __forceinline__ bool crossed(int b, int j, int st, float g, float inv, float tx, int a) {
    const int kb = st > 0 ? j : j + 1;
    const float tc = __fmul_rn(__fsub_rn((float)kb, g), inv);
    return tc < tx || (tc == tx && b < a);
}

// Cone-traced radiance of one direction from origin o; 0 on a miss.
__device__ float trace_cell(const TraceArgs& T, const Node* s_nodes, const float o[3], const float3 dv,
                            uint32_t* status) {
    const int D = T.D;
    const int res = 1 << D;
    const float fres = (float)res;
    const float d[3] = {dv.x, dv.y, dv.z};
    float g[3], dsc[3], inv[3];
    int st[3];
    bool mv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g[a] = __fmul_rn(__fsub_rn(o[a], T.lo[a]), T.scale);
        dsc[a] = __fmul_rn(d[a], T.scale);
        mv[a] = d[a] != 0.0f;
        inv[a] = mv[a] ? __fdiv_rn(1.0f, dsc[a]) : 0.0f;
        st[a] = d[a] > 0.0f ? 1 : -1;
    }
    int cell[3];
    float t = 0.0f;
    const bool inside = (g[0] >= 0.0f) && (g[0] <= fres) && (g[1] >= 0.0f) && (g[1] <= fres) &&
                        (g[2] >= 0.0f) && (g[2] <= fres);
    if (inside) {
#pragma unroll
        for (int a = 0; a < 3; ++a) cell[a] = min((int)g[a], res - 1);
    } else {
        float tn = 0.0f, tf = __int_as_float(0x7f800000);
        int enter = -1;
        for (int a = 0; a < 3; ++a) {
            if (!mv[a]) {
                if (!(g[a] >= 0.0f && g[a] <= fres)) return 0.0f;
                continue;
            }
            const float t0 = __fmul_rn(__fsub_rn(0.0f, g[a]), inv[a]);
            const float t1 = __fmul_rn(__fsub_rn(fres, g[a]), inv[a]);
            const float lo_t = (t1 < t0) ? t1 : t0;
            const float hi_t = (t0 < t1) ? t1 : t0;
            if (lo_t > tn) {
                tn = lo_t;
                enter = a;
            }
            tf = (hi_t < tf) ? hi_t : tf;
        }
        if (!(tn <= tf)) return 0.0f;
        t = tn;
        for (int a = 0; a < 3; ++a) {
            if (a == enter) {
                cell[a] = st[a] > 0 ? 0 : res - 1;
            } else {
                const float p = __fadd_rn(g[a], __fmul_rn(tn, dsc[a]));
                const int c = (p >= 0.0f) ? (int)p : 0;
                cell[a] = min(c, res - 1);
            }
        }
    }
    const float INF = __int_as_float(0x7f800000);
    const int cap = 3 * res + 16;
    bool hit = false;
    for (int it = 0; it < cap; ++it) {
        // deepest existing node holding the current cell
        uint32_t node = 0;
        int l = 0;
        while (l < D) {
            const Node nd = load_node(T, s_nodes, node);
            const int k = child_slot(cell, l, D);
            if (!((nd.mask >> k) & 1u)) break;
            node = child_id(nd, k);
            ++l;
        }
        int sl;
        if (l == D) {
            if (t >= T.t_skip) {
                hit = true;
                break;
            }
            sl = 0;
        } else {
            sl = D - l - 1;  // the empty child block at level l + 1
        }
        const int size = 1 << sl;
        int base[3];
        float te[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            base[a] = (cell[a] >> sl) << sl;
            const int kb = st[a] > 0 ? base[a] + size : base[a];
            te[a] = mv[a] ? __fmul_rn(__fsub_rn((float)kb, g[a]), inv[a]) : INF;
        }
        const int a = (te[0] <= te[1] && te[0] <= te[2]) ? 0 : (te[1] <= te[2] ? 1 : 2);
        const float tx = te[a];
        if (tx == INF) return 0.0f;
        int nc[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) {
                nc[b] = st[b] > 0 ? base[b] + size : base[b] - 1;
            } else if (!mv[b] || size == 1) {
                nc[b] = cell[b];
            } else {
                const int lo_b = base[b], hi_b = base[b] + size - 1;
                const float est = g[b] + tx * dsc[b];
                int j = (int)floorf(est);
                j = max(lo_b, min(hi_b, j));
                if (st[b] > 0) {
                    j = max(j, cell[b]);
                    while (j < hi_b && crossed(b, j + 1, 1, g[b], inv[b], tx, a)) ++j;
                    while (j > cell[b] && !crossed(b, j, 1, g[b], inv[b], tx, a)) --j;
                } else {
                    j = min(j, cell[b]);
                    while (j > lo_b && crossed(b, j - 1, -1, g[b], inv[b], tx, a)) --j;
                    while (j < cell[b] && !crossed(b, j, -1, g[b], inv[b], tx, a)) ++j;
                }
                nc[b] = j;
            }
        }
        t = tx;
        cell[0] = nc[0];
        cell[1] = nc[1];
        cell[2] = nc[2];
        if (nc[a] < 0 || nc[a] >= res) return 0.0f;
    }
    if (!hit) {
        atomicOr(status, (uint32_t)WFPG_STATUS_TRACE_CAP);
        return 0.0f;
    }
    // Eq. 6: footprint A = t^2 * omega; level whose squared side is closest
    const float A = __fmul_rn(__fmul_rn(t, t), T.omega);
    float side = T.S;
    int best = 0;
    float bd = INF;
    for (int l = 0; l <= D; ++l) {
        const float diff = fabsf(__fsub_rn(__fmul_rn(side, side), A));
        if (diff <= bd) {
            bd = diff;
            best = l;
        }
        side = __fmul_rn(side, 0.5f);
    }
    uint32_t node = 0;
    for (int l = 0; l < best; ++l) node = child_id(load_node(T, s_nodes, node), child_slot(cell, l, D));
    const float4 N = T.normal[node];
    const float2 V = T.value[node];
    const float dd = __fadd_rn(__fadd_rn(__fmul_rn(N.x, d[0]), __fmul_rn(N.y, d[1])), __fmul_rn(N.z, d[2]));
    float L = (dd <= 0.0f) ? V.x : V.y;  // the side facing back along the ray
    if (T.cos_weight) L = __fmul_rn(L, fabsf(dd));
    return L;
}

// inclusive scan of a row of N floats in warp order (chunks of 32: rounds
// k = 1, 2, 4, 8, 16 of x[i] += x[i-k], later chunks add the running total),
// then a running maximum (exact; keeps the CDF non-decreasing under rounding)
__device__ __forceinline__ float warp_scan_row(const float* src, float* dst, int N, int lane) {
    const int W = N < 32 ? N : 32;
    float carry = 0.0f, mx = 0.0f;
    for (int c0 = 0; c0 < N; c0 += W) {
        float x = lane < W ? src[c0 + lane] : 0.0f;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, x, k);
            if (k < W && lane >= k) x = __fadd_rn(x, y);
        }
        if (c0 > 0) x = __fadd_rn(carry, x);
        carry = __shfl_sync(0xffffffffu, x, W - 1);
        // running max: chunk-local max-scan then the previous chunk's max
        float m = x;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, m, k);
            if (lane >= k) m = fmaxf(m, y);
        }
        if (c0 > 0) m = fmaxf(m, mx);
        mx = __shfl_sync(0xffffffffu, m, W - 1);
        if (lane < W) dst[c0 + lane] = m;
    }
    return mx;
}

__global__ void __launch_bounds__(kGuideThreads) k_guide_build(TraceArgs T, GuideArgs G, const float* __restrict__ pos,
                                                               const uint32_t* __restrict__ origin_ray,
                                                               const uint32_t* __restrict__ n_bins_dev,
                                                               uint32_t bin_cap, float* __restrict__ pdf,
                                                               float* __restrict__ cdf_row,
                                                               float* __restrict__ cdf_marg, uint32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    Node* s_nodes = reinterpret_cast<Node*>(smem);
    const int N = G.N, NN = N * N;
    float* field = reinterpret_cast<float*>(smem + sizeof(Node) * T.smem_nodes);
    float* tmp = field + NN;
    float* rowtot = tmp + NN;
    float* marg = rowtot + N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kGuideThreads / 32;
    for (uint32_t i = tid; i < T.smem_nodes; i += kGuideThreads) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(T.node) + i);
        s_nodes[i].first_child = v.x;
        s_nodes[i].mask = v.y;
    }
    __syncthreads();
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const float tn = __fdiv_rn(2.0f, (float)N);
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint32_t r = origin_ray ? origin_ray[b] : b;
        float o[3];
        if (r == kNone) {
            o[0] = o[1] = o[2] = __int_as_float(0x7fc00000);  // no origin: every cell misses
        } else {
            o[0] = pos[3 * (size_t)r + 0];
            o[1] = pos[3 * (size_t)r + 1];
            o[2] = pos[3 * (size_t)r + 2];
        }
        const uint64_t jseed = purpose(G.seed, kJitterPurpose);
        const uint64_t jstream = bin_stream(G.frame, b);
        for (int c = tid; c < NN; c += kGuideThreads) {
            const int i = c % N, j = c / N;
            float x0 = 0.5f, x1 = 0.5f;
            if (G.jitter) {
                x0 = uniform01(jseed, jstream, 2ull * c);
                x1 = uniform01(jseed, jstream, 2ull * c + 1);
            }
            const float u = __fsub_rn(__fmul_rn(__fadd_rn((float)i, x0), tn), 1.0f);
            const float v = __fsub_rn(__fmul_rn(__fadd_rn((float)j, x1), tn), 1.0f);
            const float3 d = octa_to_dir(u, v);
            const float L = (r == kNone) ? 0.0f : trace_cell(T, s_nodes, o, d, status);
            field[c] = __fadd_rn(G.eps, L);
        }
        __syncthreads();
        if (G.blur) {
            for (int c = tid; c < NN; c += kGuideThreads) {
                const int i = c % N, j = c / N;
                const float up = (j > 0) ? field[(j - 1) * N + i] : field[N - 1 - i];
                const float dn = (j < N - 1) ? field[(j + 1) * N + i] : field[(N - 1) * N + (N - 1 - i)];
                const float m = field[c];
                tmp[c] = __fmul_rn(__fadd_rn(__fadd_rn(up, dn), __fadd_rn(m, m)), 0.25f);
            }
            __syncthreads();
            for (int c = tid; c < NN; c += kGuideThreads) {
                const int i = c % N, j = c / N;
                const float lf = (i > 0) ? tmp[c - 1] : tmp[(N - 1 - j) * N];
                const float rt = (i < N - 1) ? tmp[c + 1] : tmp[(N - 1 - j) * N + (N - 1)];
                const float m = tmp[c];
                field[c] = __fmul_rn(__fadd_rn(__fadd_rn(lf, rt), __fadd_rn(m, m)), 0.25f);
            }
            __syncthreads();
        }
        // row CDFs (one warp per row) into tmp, row totals into rowtot
        for (int j = warp; j < N; j += kWarps) {
            const float tot = warp_scan_row(field + j * N, tmp + j * N, N, lane);
            if (lane == 0) rowtot[j] = tot;
        }
        __syncthreads();
        if (warp == 0) warp_scan_row(rowtot, marg, N, lane);
        __syncthreads();
        const float den = __fmul_rn(marg[N - 1], kFourPi);
        const float nn = (float)NN;
        float* gp = pdf + (size_t)b * NN;
        float* gc = cdf_row + (size_t)b * NN;
        for (int c = tid; c < NN; c += kGuideThreads) {
            gp[c] = __fdiv_rn(__fmul_rn(field[c], nn), den);
            gc[c] = tmp[c];
        }
        for (int j = tid; j < N; j += kGuideThreads) cdf_marg[(size_t)b * N + j] = marg[j];
        __syncthreads();
    }
}

// first index with x[i] > t (N if none); x is non-decreasing
__device__ __forceinline__ int upper_bound_f(const float* __restrict__ x, int N, float t) {
    int lo = 0, hi = N;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(x + mid) > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ float clamp01(float x) {
    if (!(x >= 0.0f)) return 0.0f;
    return x >= 1.0f ? kOneMinus : x;
}

__global__ void __launch_bounds__(256) k_guide_sample(const float* __restrict__ pdf, const float* __restrict__ cdf_row,
                                                      const float* __restrict__ cdf_marg, int N, uint32_t bin_cap,
                                                      const uint32_t* __restrict__ bin_of_ray,
                                                      const float2* __restrict__ u, uint32_t n, float* __restrict__ dir,
                                                      float* __restrict__ pdf_out, uint32_t* __restrict__ cell) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = bin_of_ray[i];
    if (b >= bin_cap) {
        dir[3 * (size_t)i + 0] = dir[3 * (size_t)i + 1] = dir[3 * (size_t)i + 2] = 0.0f;
        pdf_out[i] = 0.0f;
        cell[i] = kNone;
        return;
    }
    const float2 uu = u[i];
    const float* M = cdf_marg + (size_t)b * N;
    const float t0 = __fmul_rn(uu.x, __ldg(M + N - 1));
    const int r = min(upper_bound_f(M, N, t0), N - 1);
    const float* C = cdf_row + ((size_t)b * N + r) * N;
    const float t1 = __fmul_rn(uu.y, __ldg(C + N - 1));
    const int c = min(upper_bound_f(C, N, t1), N - 1);
    const float mlo = r > 0 ? __ldg(M + r - 1) : 0.0f, mhi = __ldg(M + r);
    const float clo = c > 0 ? __ldg(C + c - 1) : 0.0f, chi = __ldg(C + c);
    const float beta = clamp01(__fdiv_rn(__fsub_rn(t0, mlo), __fsub_rn(mhi, mlo)));
    const float alpha = clamp01(__fdiv_rn(__fsub_rn(t1, clo), __fsub_rn(chi, clo)));
    const float tn = __fdiv_rn(2.0f, (float)N);
    const float su = __fsub_rn(__fmul_rn(__fadd_rn((float)c, alpha), tn), 1.0f);
    const float sv = __fsub_rn(__fmul_rn(__fadd_rn((float)r, beta), tn), 1.0f);
    const float3 d = octa_to_dir(su, sv);
    dir[3 * (size_t)i + 0] = d.x;
    dir[3 * (size_t)i + 1] = d.y;
    dir[3 * (size_t)i + 2] = d.z;
    pdf_out[i] = __ldg(pdf + (size_t)b * N * N + r * N + c);
    cell[i] = (uint32_t)(r * N + c);
}

__global__ void __launch_bounds__(256) k_guide_eval(const float* __restrict__ pdf, int N, uint32_t bin_cap,
                                                    const uint32_t* __restrict__ bin, const float* __restrict__ dir,
                                                    uint32_t n, float* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = bin[i];
    if (b >= bin_cap) {
        out[i] = 0.0f;
        return;
    }
    const float2 uv = dir_to_octa(dir[3 * (size_t)i + 0], dir[3 * (size_t)i + 1], dir[3 * (size_t)i + 2]);
    const float hn = __fmul_rn((float)N, 0.5f);
    const float a = __fmul_rn(__fadd_rn(uv.x, 1.0f), hn), c = __fmul_rn(__fadd_rn(uv.y, 1.0f), hn);
    int ii = (a >= 0.0f) ? (int)a : 0;
    int jj = (c >= 0.0f) ? (int)c : 0;
    ii = min(ii, N - 1);
    jj = min(jj, N - 1);
    out[i] = __ldg(pdf + (size_t)b * N * N + jj * N + ii);
}

// ---------------------------------------------------------------------------
static size_t guide_smem_bytes(uint32_t smem_nodes, int N) {
    return sizeof(Node) * smem_nodes + sizeof(float) * (2 * (size_t)N * N + 2 * (size_t)N);
}

int guide_build_impl(const wfpg_svo* s, const float* pos, const uint32_t* origin_ray, const uint32_t* n_bins_dev,
                     uint32_t bin_cap, const wfpg_guide_params* p, float* pdf, float* cdf_row, float* cdf_marg,
                     cudaStream_t st) {
    if (bin_cap == 0) return WFPG_OK;
    TraceArgs T;
    T.node = s->node;
    T.normal = s->normal;
    T.value = s->value;
    T.D = s->D;
    for (int a = 0; a < 3; ++a) T.lo[a] = s->lo[a];
    T.scale = s->scale;
    T.S = s->S;
    T.t_skip = p->t_skip;
    T.omega = kFourPi / (float)(p->N * p->N);
    T.cos_weight = p->cos_weight;
    const int top = s->D < kSmemTopLevels ? s->D : kSmemTopLevels;
    T.smem_nodes = s->level_off[top + 1];
    GuideArgs G;
    G.N = p->N;
    G.eps = p->eps;
    G.jitter = p->jitter;
    G.blur = p->blur;
    G.seed = p->seed;
    G.frame = p->frame;
    const size_t smem = guide_smem_bytes(T.smem_nodes, p->N);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_guide_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return WFPG_ERR_CUDA;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_guide_build, kGuideThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const uint32_t grid = min((uint64_t)bin_cap, (uint64_t)sms * per_sm);
    WFPG_LAUNCH(k_guide_build, grid, kGuideThreads, smem, st, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row,
                                                     cdf_marg, s->status);
    return cudaGetLastError() == cudaSuccess ? WFPG_OK : WFPG_ERR_CUDA;
}

int guide_sample_impl(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                      const uint32_t* bin_of_ray, const float* u, uint32_t n, float* dir, float* pdf_out,
                      uint32_t* cell, cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_guide_sample, div_up(n, 256), 256, 0, st, pdf, cdf_row, cdf_marg, N, bin_cap, bin_of_ray,
                                                   reinterpret_cast<const float2*>(u), n, dir, pdf_out, cell);
    return cudaGetLastError() == cudaSuccess ? WFPG_OK : WFPG_ERR_CUDA;
}

int guide_eval_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* bin, const float* dir, uint32_t n,
                    float* out, cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_guide_eval, div_up(n, 256), 256, 0, st, pdf, N, bin_cap, bin, dir, n, out);
    return cudaGetLastError() == cudaSuccess ? WFPG_OK : WFPG_ERR_CUDA;
}

}  // namespace wfpg
