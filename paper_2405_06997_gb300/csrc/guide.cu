// GuideRays (Alg. 3): per-bin cone-traced radiance field (Sec. 3.3, Eq. 6),
// epsilon floor, blur, warp-scan CDFs and PDF (Sec. 3.5), then inverse-CDF
// sampling and PDF evaluation for MIS.
//
// One CTA owns one bin at a time (persistent over bins): its threads march
// the N x N cell rays through the SVO -- the top levels staged in shared
// memory, deeper nodes read as 8-byte records through the read-only path --
// the field, its blur and its scans stay in shared memory, and only the
// finished pdf / cdf_row / cdf_marg rows go to global memory (or, in the fused
// variant, only the directions and densities of the bin's own rays).
//
// The SVO march returns exactly the leaf that a leaf-by-leaf 3D DDA returns:
// every boundary time is evaluated afresh as (k - g) / (d * 2^D / S) for an
// integer boundary k; when the walk sits in an empty block it jumps to the
// block's exit crossing (the smallest face time, ties x < y < z) and sets the
// other coordinates to the cells a leaf-by-leaf walk would have reached by
// that crossing (crossings earlier in (time, axis) order).
#include <algorithm>

#include <type_traits>

#include "common.cuh"
#include "march.cuh"
#include "sort.cuh"
#include "svo.cuh"

namespace wfpg {

constexpr float kOneMinus = 0x1.fffffep-1f;
constexpr int kGuideChunk = 512;   // cells whose directions are staged in shared memory at once
// default threads per bin (measured on the 1080p frame workload, GB300): 64
// with staged directions for N <= 16, 128 for N = 32, 256 above, unstaged
constexpr int kGuideDefaultThreadsSmall = 64, kGuideDefaultThreadsMid = 128, kGuideDefaultThreadsLarge = 256;
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
    const uint32_t* top;  // the SVO's top index (levels 0 .. G), NULL when it has none
    int G;                // deepest indexed level, -1 without an index
    uint32_t top_offG;    // offset of level G's grid in the top index
    const uint32_t* occ;  // occupancy bitmaps of levels G + 1 .. D (NULL: none)
    uint32_t occ_off[kOccMaxDepth - kTopLevelMax];  // word offsets of levels G + 1, G + 2, ...
    int flat;             // 1: the index and the bitmaps give every cell's deepest level directly
};

// depth D and index depth G of the SVO: compile-time constants in a kernel
// specialised on the depth (kD > 0; the index then covers levels 0 .. min(kD, 6)),
// else read from T
template <int kD>
__device__ __forceinline__ int svo_depth(const TraceArgs& T) {
    return kD > 0 ? kD : T.D;
}
template <int kD>
__device__ __forceinline__ int index_depth(const TraceArgs& T) {
    return kD > 0 ? (kD < kTopLevelMax ? kD : kTopLevelMax) : T.G;
}

// offset of level l's grid in the top index: 8^0 + ... + 8^(l-1) = (8^l - 1) / 7
__device__ __forceinline__ uint32_t top_offset(int l) { return ((1u << (3 * l)) - 1u) / 7u; }
// the top index's entry of leaf cell (cx, cy, cz) at level l: (level << 28) | node
template <int kD = 0>
__device__ __forceinline__ uint32_t top_entry(const TraceArgs& T, int l, int cx, int cy, int cz) {
    const int sh = svo_depth<kD>(T) - l;
    const uint32_t i = ((uint32_t)(cz >> sh) << (2 * l)) | ((uint32_t)(cy >> sh) << l) | (uint32_t)(cx >> sh);
    return __ldg(T.top + top_offset(l) + i);
}

// bits 0 .. 9 of v moved to bits 0, 3, 6, ..., 27 (one coordinate of a Morton key)
__device__ __forceinline__ uint32_t spread3_10(uint32_t v) {
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// the deepest existing level below the index from the bitmaps, with Morton keys of type Key
template <typename Key>
__device__ __forceinline__ int bitmap_level(const TraceArgs& T, int D, int G, Key key) {
    uint32_t w[kOccMaxDepth - kTopLevelMax];
#pragma unroll
    for (int j = 0; j < kOccMaxDepth - kTopLevelMax; ++j) {
        const int l = G + 1 + j;
        w[j] = 0u;
        if (l <= D) w[j] = __ldg(T.occ + T.occ_off[j] + (uint32_t)((key >> (3 * (D - l))) >> 5));
    }
    int L = G;
#pragma unroll
    for (int j = 0; j < kOccMaxDepth - kTopLevelMax; ++j) {
        const int l = G + 1 + j;
        if (l > D) break;
        // a select rather than an early exit: every lane runs the same few iterations
        if (L == l - 1 && ((w[j] >> (uint32_t)((key >> (3 * (D - l))) & 31u)) & 1u)) L = l;
    }
    return L;
}

// Deepest level holding an existing node that contains leaf cell (cx, cy, cz),
// when the index and the bitmaps cover every level (T.flat): the index gives
// it down to level G, one bit per deeper level the rest; the loads are
// independent of one another.
template <int kD = 0>
__device__ __forceinline__ int deepest_level(const TraceArgs& T, int cx, int cy, int cz) {
    const int D = svo_depth<kD>(T), G = index_depth<kD>(T);
    const int sh = D - G;
    const uint32_t ti =
        ((uint32_t)(cz >> sh) << (2 * G)) | ((uint32_t)(cy >> sh) << G) | (uint32_t)(cx >> sh);
    const int L0 = (int)(__ldg(T.top + T.top_offG + ti) >> 28);
    // the Morton key (x bits at 3i, y at 3i + 1, z at 3i + 2) of the leaf cell: 32 bits up to
    // depth 10 (the flat walk of a kernel not specialised on the depth stops there), 64 bits at 11
    if constexpr (kD > 10) {
        const uint64_t key = morton3((uint32_t)cx, (uint32_t)cy, (uint32_t)cz);
        const int L = bitmap_level<uint64_t>(T, D, G, key);
        return L0 < G ? L0 : L;
    }
    const uint32_t key =
        spread3_10((uint32_t)cx) | (spread3_10((uint32_t)cy) << 1) | (spread3_10((uint32_t)cz) << 2);
    const int L = bitmap_level<uint32_t>(T, D, G, key);
    return L0 < G ? L0 : L;
}

struct GuideArgs {
    int N;
    float eps;
    int jitter;
    int blur;
    uint64_t seed;
    uint32_t frame;
    const uint32_t* frame_dev;  // when set, the frame index is read from device memory
};

// fused sampling: after a bin's CDF is built in shared memory, every ray of the
// bin draws its next direction from alpha * field + (1 - alpha) * cosine.  A bin
// with more than `split` rays copies its field and CDFs to a spill slot instead,
// and k_spill_sample draws its rays with the whole GPU (same arithmetic).
struct FusedArgs {
    const uint32_t* ray_order;
    const uint32_t* bin_offset;
    const float* nrm;   // xyz per ray
    const float* u;     // 3 uniforms per ray: two for the direction, one for the mixture choice
    float alpha;
    float* dir;         // xyz per ray
    float* pdf;         // mixture density per ray
    uint32_t split;     // 0: never spill
    uint32_t spill_cap;
    unsigned long long* spill_ctr;  // (slots << 40) | chunks, appended together
    uint32_t* spill_bin;            // bin of each slot
    uint32_t* spill_base;           // first chunk of each slot
    float* spill_tab;               // per slot: field (N^2), row CDFs (N^2), marginal (N)
    const float* eval_dir;          // optional: a second direction per ray (e.g. a light sample) whose
    float* eval_pdf;                // mixture density is written here, from the same field
};
constexpr int kSpillChunk = 256;  // rays per block-iteration of k_spill_sample
constexpr unsigned long long kSpillChunkMask = (1ull << 40) - 1;

__device__ __forceinline__ Node load_node(const TraceArgs& T, const Node* s_nodes, uint32_t id) {
    if (id < T.smem_nodes) return s_nodes[id];
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(T.node) + id);
    Node n;
    n.first_child = v.x;
    n.mask = v.y;
    return n;
}

// the node at level l (>= G) holding leaf cell (cx, cy, cz), which must exist:
// from the index's node at level G, descending l - G levels
template <int kD = 0>
__device__ __forceinline__ uint32_t node_at_level(const TraceArgs& T, const Node* s_nodes, int l, int cx, int cy,
                                                  int cz) {
    const int D = svo_depth<kD>(T), G = index_depth<kD>(T);
    uint32_t node = top_entry<kD>(T, G, cx, cy, cz) & kTopNodeMask;
    for (int lv = G; lv < l; ++lv) {
        const Node nd = load_node(T, s_nodes, node);
        const int sh = D - 1 - lv;
        const int k = ((cx >> sh) & 1) | (((cy >> sh) & 1) << 1) | (((cz >> sh) & 1) << 2);
        node = child_id(nd, k);
    }
    return node;
}

// first index with x[i] > t (N if none) in a non-decreasing shared-memory row
__device__ __forceinline__ int upper_bound_s(const float* x, int N, float t) {
    int lo = 0, hi = N;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (x[mid] > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ float clamp_unit(float x) {
    if (!(x >= 0.0f)) return 0.0f;
    return x >= 1.0f ? kOneMinus : x;
}

// inverse-CDF sample of the piecewise-constant field (row CDFs C, marginal M,
// all in shared memory); returns the direction and the chosen cell's field
// value (same arithmetic as guide_sample)
__device__ __forceinline__ float3 sample_cdf(const float* f, const float* C, const float* M, int N, float u0,
                                             float u1, float tn, float* fcell) {
    const float t0 = __fmul_rn(u0, M[N - 1]);
    const int r = min(upper_bound_s(M, N, t0), N - 1);
    const float* Cr = C + r * N;
    const float t1 = __fmul_rn(u1, Cr[N - 1]);
    const int c = min(upper_bound_s(Cr, N, t1), N - 1);
    const float mlo = r > 0 ? M[r - 1] : 0.0f, mhi = M[r];
    const float clo = c > 0 ? Cr[c - 1] : 0.0f, chi = Cr[c];
    const float beta = clamp_unit(__fdiv_rn(__fsub_rn(t0, mlo), __fsub_rn(mhi, mlo)));
    const float alpha = clamp_unit(__fdiv_rn(__fsub_rn(t1, clo), __fsub_rn(chi, clo)));
    const float su = __fsub_rn(__fmul_rn(__fadd_rn((float)c, alpha), tn), 1.0f);
    const float sv = __fsub_rn(__fmul_rn(__fadd_rn((float)r, beta), tn), 1.0f);
    *fcell = f[r * N + c];
    return octa_to_dir(su, sv);
}



// one ray of the one-sample mixture: guided (inverse CDF) if u2 < alpha, else
// cosine about the normal; writes the direction and the mixture density
__device__ __forceinline__ void sample_ray(const FusedArgs& F, uint32_t ray, const float* f, const float* C,
                                           const float* M, int N, float nn, float den, float tn) {
    const float u0 = F.u[3 * (size_t)ray], u1 = F.u[3 * (size_t)ray + 1], u2 = F.u[3 * (size_t)ray + 2];
    const float nx = F.nrm[3 * (size_t)ray], ny = F.nrm[3 * (size_t)ray + 1], nz = F.nrm[3 * (size_t)ray + 2];
    float3 d;
    float pg;
    if (u2 < F.alpha) {
        d = sample_cdf(f, C, M, N, u0, u1, tn, &pg);
        pg = __fdiv_rn(__fmul_rn(pg, nn), den);
    } else {
        d = cosine_dir(nx, ny, nz, u0, u1);
        pg = __fdiv_rn(__fmul_rn(f[octa_cell(d, N)], nn), den);
    }
    const float cs = fmaxf(0.0f, nx * d.x + ny * d.y + nz * d.z);
    F.dir[3 * (size_t)ray] = d.x;
    F.dir[3 * (size_t)ray + 1] = d.y;
    F.dir[3 * (size_t)ray + 2] = d.z;
    F.pdf[ray] = F.alpha * pg + (1.0f - F.alpha) * cs * 0.31830988618379067f;
    if (F.eval_dir) {
        const float3 e = make_float3(F.eval_dir[3 * (size_t)ray], F.eval_dir[3 * (size_t)ray + 1],
                                     F.eval_dir[3 * (size_t)ray + 2]);
        const float pe = __fdiv_rn(__fmul_rn(f[octa_cell(e, N)], nn), den);
        const float ce = fmaxf(0.0f, nx * e.x + ny * e.y + nz * e.z);
        F.eval_pdf[ray] = F.alpha * pe + (1.0f - F.alpha) * ce * 0.31830988618379067f;
    }
}

// rays of the spilled bins, kSpillChunk per block-iteration, tables read from
// global memory (L2); chunk c belongs to the last slot whose first chunk <= c
__global__ void __launch_bounds__(kSpillChunk) k_spill_sample(FusedArgs F, int N) {
    const unsigned long long ctr = *F.spill_ctr;
    const uint32_t nslots = min((uint32_t)(ctr >> 40), F.spill_cap);
    const uint32_t nch = (uint32_t)(ctr & kSpillChunkMask);
    if (nslots == 0) return;
    const int NN = N * N;
    const float nn = (float)NN, tn = __fdiv_rn(2.0f, (float)N);
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        uint32_t lo = 0, hi = nslots;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (F.spill_base[mid] <= c) lo = mid;
            else hi = mid;
        }
        const uint32_t b = F.spill_bin[lo];
        const uint32_t k = F.bin_offset[b] + (c - F.spill_base[lo]) * kSpillChunk + threadIdx.x;
        if (k >= F.bin_offset[b + 1]) continue;
        const float* tab = F.spill_tab + (size_t)lo * (2 * NN + N);
        const float den = __fmul_rn(tab[2 * NN + N - 1], kFourPi);
        sample_ray(F, F.ray_order[k], tab, tab + NN, tab + 2 * NN, N, nn, den, tn);
    }
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

// kGuideThreads threads work on one bin at a time; kStage: the chunk's cone
// directions are computed by all threads together into shared memory before
// the march (otherwise each lane computes its ray's direction when it takes it)
constexpr int kDescentPerPass = 4;  // SVO levels a lane descends per pass of the walk loop
constexpr int kWbWords = 11;  // per buffered ray: cell, d (3), 1/(d 2^D/S) (3), t, start cell (3)

// direction of cell c (jittered point or centre) and its per-axis reciprocal
// 1 / (d 2^D / S) (0 on an axis the ray does not move along)
__device__ __forceinline__ void cell_ray(const TraceArgs& T, const GuideArgs& G, int c, uint64_t jseed,
                                         uint64_t jstream, float tn, float3* d, float3* iv) {
    const int N = G.N;
    const int i = c % N, j = c / N;
    float x0 = 0.5f, x1 = 0.5f;
    if (G.jitter) {
        x0 = uniform01(jseed, jstream, 2ull * c);
        x1 = uniform01(jseed, jstream, 2ull * c + 1);
    }
    const float u = __fsub_rn(__fmul_rn(__fadd_rn((float)i, x0), tn), 1.0f);
    const float v = __fsub_rn(__fmul_rn(__fadd_rn((float)j, x1), tn), 1.0f);
    *d = octa_to_dir(u, v);
    iv->x = d->x != 0.0f ? __fdiv_rn(1.0f, __fmul_rn(d->x, T.scale)) : 0.0f;
    iv->y = d->y != 0.0f ? __fdiv_rn(1.0f, __fmul_rn(d->y, T.scale)) : 0.0f;
    iv->z = d->z != 0.0f ? __fdiv_rn(1.0f, __fmul_rn(d->z, T.scale)) : 0.0f;
}

// start of a cone ray: the cell holding the origin (or the slab entry into the
// grid box, with its entry time), then every crossing strictly before t_skip
// taken at once (no cell entered before t_skip can be the hit).  False if the
// ray never reaches a cell at t_skip inside the grid.
__device__ __forceinline__ bool ray_start(const TraceArgs& T, bool has_origin, bool inside, float gx, float gy,
                                          float gz, float dx, float dy, float dz, float ivx, float ivy, float ivz,
                                          int res, float fres, float* t, int* cx, int* cy, int* cz) {
    const float INF = __int_as_float(0x7f800000);
    bool alive = has_origin;
    *t = 0.0f;
    if (alive && inside) {
        *cx = min((int)gx, res - 1);
        *cy = min((int)gy, res - 1);
        *cz = min((int)gz, res - 1);
    } else if (alive) {
        // slab entry into the grid box
        float tnr = 0.0f, tfr = INF;
        int enter = -1;
        const float gg[3] = {gx, gy, gz}, iv[3] = {ivx, ivy, ivz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (iv[a] == 0.0f) {
                if (!(gg[a] >= 0.0f && gg[a] <= fres)) alive = false;
                continue;
            }
            const float t0 = __fmul_rn(__fsub_rn(0.0f, gg[a]), iv[a]);
            const float t1 = __fmul_rn(__fsub_rn(fres, gg[a]), iv[a]);
            const float lo_t = (t1 < t0) ? t1 : t0;
            const float hi_t = (t0 < t1) ? t1 : t0;
            if (lo_t > tnr) {
                tnr = lo_t;
                enter = a;
            }
            tfr = (hi_t < tfr) ? hi_t : tfr;
        }
        if (!(tnr <= tfr)) alive = false;
        if (alive) {
            *t = tnr;
            const float dd[3] = {dx, dy, dz};
            int cc[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == enter) {
                    cc[a] = iv[a] > 0.0f ? 0 : res - 1;
                } else {
                    const float p = __fadd_rn(gg[a], __fmul_rn(tnr, __fmul_rn(dd[a], T.scale)));
                    const int c = (p >= 0.0f) ? (int)p : 0;
                    cc[a] = min(c, res - 1);
                }
            }
            *cx = cc[0];
            *cy = cc[1];
            *cz = cc[2];
        }
    }
    if (alive && *t < T.t_skip) {
        *cx = skip_before(*cx, gx, ivx, T.t_skip, res);
        *cy = skip_before(*cy, gy, ivy, T.t_skip, res);
        *cz = skip_before(*cz, gz, ivz, T.t_skip, res);
        if (*cx < 0 || *cx >= res || *cy < 0 || *cy >= res || *cz < 0 || *cz >= res) alive = false;
    }
    return alive;
}

// The cone query of a hit leaf (Eq. 6): the level whose squared side is closest
// to the footprint t^2 omega (ties to the finer level), its node holding the
// leaf, and that node's value on the side facing back along the ray.  an_path:
// the ancestor at the chosen level when it lies on the caller's node path at or
// below G (only used without the flat index).
template <int kD = 0>
__device__ __forceinline__ float hit_value(const TraceArgs& T, const Node* s_nodes, float t, int cx, int cy, int cz,
                                           float dx, float dy, float dz, const uint32_t* stk, int stride) {
    const int D = svo_depth<kD>(T), G = index_depth<kD>(T);
    const float A = __fmul_rn(__fmul_rn(t, t), T.omega);
    float side = T.S, bd = __int_as_float(0x7f800000);
    int best = 0;
    for (int l = 0; l <= D; ++l) {
        const float diff = fabsf(__fsub_rn(__fmul_rn(side, side), A));
        if (diff <= bd) {
            bd = diff;
            best = l;
        }
        side = __fmul_rn(side, 0.5f);
    }
    // the hit leaf's ancestor at that level: the top index, else the node path (or a short descent)
    const uint32_t an = best < G ? (top_entry<kD>(T, best, cx, cy, cz) & kTopNodeMask)
                                   : (T.flat ? node_at_level<kD>(T, s_nodes, best, cx, cy, cz) : stk[best * stride]);
    const float4 Nn = T.normal[an];
    const float2 V = T.value[an];
    const float dd = __fadd_rn(__fadd_rn(__fmul_rn(Nn.x, dx), __fmul_rn(Nn.y, dy)), __fmul_rn(Nn.z, dz));
    float L = (dd <= 0.0f) ? V.x : V.y;  // the side facing back along the ray
    if (T.cos_weight) L = __fmul_rn(L, fabsf(dd));
    return L;
}

constexpr int kHitQueue = 32;  // per-warp queue of hits awaiting their cone query (flat index only)
constexpr int kHitWords = 7;   // cell, t, leaf cell (x | y << 16, then z; D <= 11), direction (3)

// the cone queries of queue entries [e0, e0 + n) (n <= 32), one per lane, into out[cell]
template <int kD = 0>
__device__ __forceinline__ void flush_hits(const TraceArgs& T, const GuideArgs& G, const Node* s_nodes,
                                           const uint32_t* hq, int e0, int n, int lane, float* out) {
    if (lane < n) {
        const int e = e0 + lane;
        const int q = (int)hq[0 * kHitQueue + e];
        const float t = __uint_as_float(hq[1 * kHitQueue + e]);
        const uint32_t c = hq[2 * kHitQueue + e];
        const int cx = (int)(c & 0xffffu), cy = (int)(c >> 16), cz = (int)hq[3 * kHitQueue + e];
        const float dx = __uint_as_float(hq[4 * kHitQueue + e]), dy = __uint_as_float(hq[5 * kHitQueue + e]),
                    dz = __uint_as_float(hq[6 * kHitQueue + e]);
        out[q] = __fadd_rn(G.eps, hit_value<kD>(T, s_nodes, t, cx, cy, cz, dx, dy, dz, nullptr, 0));
    }
}

// separable [1 2 1] / 4 blur of an N x N field with the octahedral mirror at the
// edges (rows first into tmp, then columns back into field); every thread of
// the CTA calls it, with the barriers inside
__device__ __forceinline__ void blur_field(float* field, float* tmp, int N, int tid, int nthreads) {
    const int NN = N * N;
    for (int c = tid; c < NN; c += nthreads) {
        const int i = c % N, j = c / N;
        const float up = (j > 0) ? field[(j - 1) * N + i] : field[N - 1 - i];
        const float dn = (j < N - 1) ? field[(j + 1) * N + i] : field[(N - 1) * N + (N - 1 - i)];
        const float m = field[c];
        tmp[c] = __fmul_rn(__fadd_rn(__fadd_rn(up, dn), __fadd_rn(m, m)), 0.25f);
    }
    __syncthreads();
    for (int c = tid; c < NN; c += nthreads) {
        const int i = c % N, j = c / N;
        const float lf = (i > 0) ? tmp[c - 1] : tmp[(N - 1 - j) * N];
        const float rt = (i < N - 1) ? tmp[c + 1] : tmp[(N - 1 - j) * N + (N - 1)];
        const float m = tmp[c];
        field[c] = __fmul_rn(__fadd_rn(__fadd_rn(lf, rt), __fadd_rn(m, m)), 0.25f);
    }
    __syncthreads();
}

// The cone rays of cells c0 .. c0 + cn - 1 of one bin (Sec. 3.3, Eq. 6): each
// lane marches one cell's ray through the SVO, a lane whose ray ends takes the
// next cell; out[q] = eps + the cone query of cell c0 + q (shared or global
// memory).  Called by every thread of the CTA; ends with a barrier.
template <int kGuideThreads, bool kStage>
__device__ __forceinline__ void march_chunk(const TraceArgs& T, const GuideArgs& G, const Node* s_nodes,
                                            uint32_t* s_stack, float* s_ray, float* wbuf, int* s_next, int c0,
                                            int cn, int chunk, bool has_origin, bool inside, float gx, float gy,
                                            float gz, uint64_t jseed, uint64_t jstream, float tn, uint32_t* status,
                                            float* out, uint32_t* hqueue) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int D = T.D;
    const int res = 1 << D;
    const float fres = (float)res;
    const float INF = __int_as_float(0x7f800000);
    const int cap = 3 * res + 16;
    uint32_t* stk = s_stack + tid;  // this thread's node path, one entry per level (stride = block size)
    // ---- directions of this chunk's cells, computed by all threads together
    for (int q = tid; kStage && q < cn; q += kGuideThreads) {
        float3 d, iv;
        cell_ray(T, G, c0 + q, jseed, jstream, tn, &d, &iv);
        s_ray[0 * chunk + q] = d.x;
        s_ray[1 * chunk + q] = d.y;
        s_ray[2 * chunk + q] = d.z;
        s_ray[3 * chunk + q] = iv.x;
        s_ray[4 * chunk + q] = iv.y;
        s_ray[5 * chunk + q] = iv.z;
    }
    if (tid == 0) *s_next = 0;
    __syncthreads();
    // ---- cone rays: each lane marches one cell's ray; finished lanes take the next cell
    int q = -1;  // current cell of the chunk (-1: none, >= cn: no work left)
    float dx = 0.f, dy = 0.f, dz = 0.f, ivx = 0.f, ivy = 0.f, ivz = 0.f, t = 0.f;
    int cx = 0, cy = 0, cz = 0, level = 0, steps = 0;
    uint32_t node = 0;
    int wb_n = 0, wb_head = 0;  // unstaged: entries in this warp's ray buffer, next one to hand out
    bool wb_dry = false;        // unstaged: no cells of the chunk left for this warp
    float* wb = wbuf + warp * (kWbWords * 32);
    uint32_t* hq = hqueue + warp * (kHitQueue * kHitWords);
    int hq_n = 0;       // entries in this warp's hit queue
    bool pend = false;  // this lane's ray hit a leaf in the last pass and waits for the queue
    for (;;) {
        if (T.flat) {
            // hits of the last pass join the warp's queue; when it would overflow, its entries
            // get their cone queries together, nearly every lane busy
            const uint32_t hm = __ballot_sync(0xffffffffu, pend);
            if (hm) {
                if (hq_n + __popc(hm) > kHitQueue) {
                    flush_hits(T, G, s_nodes, hq, 0, hq_n, lane, out);
                    hq_n = 0;
                    __syncwarp();
                }
                if (pend) {
                    const int e = hq_n + __popc(hm & lt);
                    hq[0 * kHitQueue + e] = (uint32_t)q;
                    hq[1 * kHitQueue + e] = __float_as_uint(t);
                    hq[2 * kHitQueue + e] = (uint32_t)cx | ((uint32_t)cy << 16);
                    hq[3 * kHitQueue + e] = (uint32_t)cz;
                    hq[4 * kHitQueue + e] = __float_as_uint(dx);
                    hq[5 * kHitQueue + e] = __float_as_uint(dy);
                    hq[6 * kHitQueue + e] = __float_as_uint(dz);
                    q = -1;
                    pend = false;
                }
                hq_n += __popc(hm);
                __syncwarp();
            }
        }
        const bool idle = q < 0;
        const uint32_t need = __ballot_sync(0xffffffffu, idle);
        if (kStage) {
            if (need) {
                const int leader = __ffs(need) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(s_next, __popc(need));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (idle) {
                    q = base + __popc(need & lt);
                    if (q < cn) {
                        dx = s_ray[0 * chunk + q];
                        dy = s_ray[1 * chunk + q];
                        dz = s_ray[2 * chunk + q];
                        ivx = s_ray[3 * chunk + q];
                        ivy = s_ray[4 * chunk + q];
                        ivz = s_ray[5 * chunk + q];
                        const bool alive = ray_start(T, has_origin, inside, gx, gy, gz, dx, dy, dz, ivx, ivy,
                                                     ivz, res, fres, &t, &cx, &cy, &cz);
                        if (!alive) {
                            out[q] = __fadd_rn(G.eps, 0.0f);
                            q = -1;
                        } else {
                            node = 0;
                            level = T.G >= 0 ? -1 : 0;  // -1: enter through the top index
                            steps = 0;
                            stk[0] = 0;
                        }
                    }
                }
            }
            // leave only when every lane has run out of cells (a lane whose new ray
            // died at its start is idle again and fetches once more)
            if (__all_sync(0xffffffffu, q >= cn)) {
                if (hq_n > 0) flush_hits(T, G, s_nodes, hq, 0, hq_n, lane, out);
                break;
            }
            if (q < 0 || q >= cn) continue;  // idle, or out of cells: no ray to step
        } else {
            // the whole warp sets up the next 32 cells' rays at once (converged), so a
            // lane that finishes a ray takes a ready one instead of stalling its warp
            // on a setup of its own
            if (need && wb_head == wb_n && !wb_dry) {
                int base = 0;
                if (lane == 0) base = atomicAdd(s_next, 32);
                base = __shfl_sync(0xffffffffu, base, 0);
                wb_n = max(0, min(32, cn - base));
                wb_head = 0;
                wb_dry = wb_n == 0;
                if (lane < wb_n) {
                    const int c = c0 + base + lane;
                    float3 d, iv;
                    cell_ray(T, G, c, jseed, jstream, tn, &d, &iv);
                    float t0;
                    int x0, y0, z0;
                    const bool alive = ray_start(T, has_origin, inside, gx, gy, gz, d.x, d.y, d.z, iv.x,
                                                 iv.y, iv.z, res, fres, &t0, &x0, &y0, &z0);
                    if (!alive) out[base + lane] = __fadd_rn(G.eps, 0.0f);
                    wb[0 * 32 + lane] = __int_as_float(alive ? base + lane : -1);
                    wb[1 * 32 + lane] = d.x;
                    wb[2 * 32 + lane] = d.y;
                    wb[3 * 32 + lane] = d.z;
                    wb[4 * 32 + lane] = iv.x;
                    wb[5 * 32 + lane] = iv.y;
                    wb[6 * 32 + lane] = iv.z;
                    wb[7 * 32 + lane] = t0;
                    wb[8 * 32 + lane] = __int_as_float(x0);
                    wb[9 * 32 + lane] = __int_as_float(y0);
                    wb[10 * 32 + lane] = __int_as_float(z0);
                }
                __syncwarp();
            }
            if (need && wb_head < wb_n) {
                const int k = wb_head + __popc(need & lt);
                if (idle && k < wb_n) {
                    q = __float_as_int(wb[0 * 32 + k]);  // -1: the ray died at its start
                    dx = wb[1 * 32 + k];
                    dy = wb[2 * 32 + k];
                    dz = wb[3 * 32 + k];
                    ivx = wb[4 * 32 + k];
                    ivy = wb[5 * 32 + k];
                    ivz = wb[6 * 32 + k];
                    t = wb[7 * 32 + k];
                    cx = __float_as_int(wb[8 * 32 + k]);
                    cy = __float_as_int(wb[9 * 32 + k]);
                    cz = __float_as_int(wb[10 * 32 + k]);
                    node = 0;
                    level = T.G >= 0 ? -1 : 0;  // -1: enter through the top index
                    steps = 0;
                    stk[0] = 0;
                }
                wb_head = min(wb_n, wb_head + __popc(need));
                __syncwarp();  // entries are read before a refill overwrites them
            }
            if (wb_dry && __all_sync(0xffffffffu, q < 0)) {
                if (hq_n > 0) flush_hits(T, G, s_nodes, hq, 0, hq_n, lane, out);
                break;
            }
            if (q < 0) continue;  // idle: no ray to step
        }
        // ---- one step: deepest existing node holding the cell, then hit or skip its empty block.
        // At most kDescentPerPass levels per pass of the loop: a lane with a deeper descent
        // goes on in the next pass instead of holding its whole warp in this one
        if (level < 0) {
            if (T.flat) {
                // one step per pass: the cell's deepest existing level, then its hit or skip
                level = deepest_level(T, cx, cy, cz);
            } else {
                // the deepest existing node at a level <= G holding the cell, from the top index
                const uint32_t e = top_entry(T, T.G, cx, cy, cz);
                level = (int)(e >> 28);
                node = e & kTopNodeMask;
                stk[level * kGuideThreads] = node;
            }
        }
        bool settled = true;
        for (int dl = 0; !T.flat && level < D; ++dl) {
            if (dl == kDescentPerPass) {
                settled = false;
                break;
            }
            const Node nd = load_node(T, s_nodes, node);
            const int sh = D - 1 - level;
            const int k = ((cx >> sh) & 1) | (((cy >> sh) & 1) << 1) | (((cz >> sh) & 1) << 2);
            if (!((nd.mask >> k) & 1u)) break;
            node = child_id(nd, k);
            ++level;
            stk[level * kGuideThreads] = node;
        }
        if (!settled) continue;
        float L = 0.0f;
        bool done = false;
        if (level == D && t >= T.t_skip) {
            if (T.flat) {
                pend = true;  // its cone query waits for a full batch (queued at the next pass)
            } else {
                L = hit_value(T, s_nodes, t, cx, cy, cz, dx, dy, dz, stk, kGuideThreads);
                done = true;
            }
        } else {
            // leave the empty block (or a leaf entered before t_skip) through its first exit crossing
            const int sl = (level == D) ? 0 : D - level - 1;
            const int size = 1 << sl;
            const int bx = (cx >> sl) << sl, by = (cy >> sl) << sl, bz = (cz >> sl) << sl;
            const int ex = ivx > 0.0f ? bx + size : bx - 1;
            const int ey = ivy > 0.0f ? by + size : by - 1;
            const int ez = ivz > 0.0f ? bz + size : bz - 1;
            const float tex = ivx != 0.0f ? cross_time(ex, ivx > 0.0f, gx, ivx) : INF;
            const float tey = ivy != 0.0f ? cross_time(ey, ivy > 0.0f, gy, ivy) : INF;
            const float tez = ivz != 0.0f ? cross_time(ez, ivz > 0.0f, gz, ivz) : INF;
            const int a = (tex <= tey && tex <= tez) ? 0 : (tey <= tez ? 1 : 2);
            const float tx = a == 0 ? tex : (a == 1 ? tey : tez);
            // the two other axes p < q, gathered by selects so that every lane runs
            // the catch-up exactly twice (ties: an axis precedes the exit axis a
            // when its index is smaller)
            const int p = a == 0 ? 1 : 0, q = a == 2 ? 1 : 2;
            const int cp = p == 0 ? cx : cy, cq = q == 1 ? cy : cz;
            const int bp = p == 0 ? bx : by, bq = q == 1 ? by : bz;
            const float gp = p == 0 ? gx : gy, gq = q == 1 ? gy : gz;
            const float ip = p == 0 ? ivx : ivy, iq = q == 1 ? ivy : ivz;
            const float dp = p == 0 ? dx : dy, dq = q == 1 ? dy : dz;
            const int np = advance_axis(cp, bp, size, gp, ip, __fmul_rn(dp, T.scale), tx, p < a);
            const int nq = advance_axis(cq, bq, size, gq, iq, __fmul_rn(dq, T.scale), tx, q < a);
            const int na = a == 0 ? ex : (a == 1 ? ey : ez);
            const int nx = a == 0 ? na : np;
            const int ny = a == 1 ? na : (p == 1 ? np : nq);
            const int nz = a == 2 ? na : nq;
            if (tx == INF || na < 0 || na >= res) {
                done = true;  // left the grid: miss
            } else if (++steps > cap) {
                atomicOr(status, (uint32_t)WFPG_STATUS_TRACE_CAP);
                done = true;
            } else {
                // restart the descent from the deepest ancestor shared with the new cell, or
                // through the top index when that ancestor lies above its deepest level
                const uint32_t diff = (uint32_t)((cx ^ nx) | (cy ^ ny) | (cz ^ nz));
                const int lc = D - 1 - (31 - __clz(diff));
                if (!T.flat && lc >= T.G) {
                    level = lc;
                    node = stk[lc * kGuideThreads];
                } else {
                    level = -1;
                }
                cx = nx;
                cy = ny;
                cz = nz;
                t = tx;
            }
        }
        if (done) {
            out[q] = __fadd_rn(G.eps, L);
            q = -1;
        }
    }
    __syncthreads();
}

// 1024 resident threads per SM (32 warps): up to 64 registers a thread.  The
// walk is issue-bound, and 64 registers (fewer recomputed values) beat 48
// registers with 40 warps on the GB300; the fused variant gets the same budget
template <int kGuideThreads, bool kStage, bool kFused, bool kSplit>
__global__ void __launch_bounds__(kGuideThreads, 1024 / kGuideThreads) k_guide_build(TraceArgs T, GuideArgs G, FusedArgs F,
                                                               const float* __restrict__ pos,
                                                               const uint32_t* __restrict__ origin_ray,
                                                               const uint32_t* __restrict__ n_bins_dev,
                                                               uint32_t bin_cap, float* __restrict__ pdf,
                                                               float* __restrict__ cdf_row,
                                                               float* __restrict__ cdf_marg, uint32_t* status,
                                                               uint32_t* __restrict__ bin_next, int parts_arg,
                                                               uint32_t slots) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = G.N, NN = N * N;
    const int D = T.D;
    const int chunk = kStage ? (NN < kGuideChunk ? NN : kGuideChunk) : NN;
    Node* s_nodes = reinterpret_cast<Node*>(smem);
    uint32_t* s_stack = reinterpret_cast<uint32_t*>(smem + sizeof(Node) * T.smem_nodes);
    float* s_ray = reinterpret_cast<float*>(s_stack + (D + 1) * kGuideThreads);  // 6 x chunk: d, 1/(d 2^D/S)
    float* wbuf = s_ray;  // unstaged: per warp, kWbWords x 32 entries of ready rays
    uint32_t* hqueue = reinterpret_cast<uint32_t*>(s_ray + (kStage ? 6 * chunk : (kGuideThreads / 32) * kWbWords * 32));
    float* field = reinterpret_cast<float*>(hqueue + (kGuideThreads / 32) * kHitQueue * kHitWords);
    float* tmp = field + NN;
    float* rowtot = tmp + NN;
    float* marg = rowtot + N;
    __shared__ int s_next;
    __shared__ uint32_t s_slot;
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
    const int res = 1 << D;
    const float fres = (float)res;
    const float INF = __int_as_float(0x7f800000);
    // Work units are (bin, part): the cells of a bin are split over `parts` CTAs
    // (1 for the fused call); the CTA that completes a bin's last part gathers its
    // field and finishes the bin.  Units are taken dynamically: the first by CTA
    // index, the next from a counter (zeroed before the launch) as each CTA
    // finishes one, so that cheap and expensive units even out.  By default a bin
    // is split only while its parts still fit in one wave of resident CTAs: with
    // few bins the idle SMs take parts of them; with a wave of bins or more,
    // splitting only adds each part's tail.
    int parts = (kFused || !kSplit) ? 1 : parts_arg;
    if (kSplit && !kFused && parts == 0) {
        parts = 1;
        while (parts < 8 && (uint64_t)nb * (uint64_t)(2 * parts) <= slots) parts *= 2;
    }
    const int part_cells = NN / parts;
    const uint32_t n_units = nb * (uint32_t)parts;
    __shared__ uint32_t s_unit;
    __shared__ int s_last;
    for (uint32_t u = blockIdx.x; u < n_units;) {
        const uint32_t b = u / (uint32_t)parts;
        const int cbeg = (int)(u % (uint32_t)parts) * part_cells, cend = cbeg + part_cells;
        const uint32_t r = origin_ray ? origin_ray[b] : b;
        float ox = 0.0f, oy = 0.0f, oz = 0.0f;
        if (r != kNone) {
            ox = pos[3 * (size_t)r + 0];
            oy = pos[3 * (size_t)r + 1];
            oz = pos[3 * (size_t)r + 2];
        }
        const float gx = __fmul_rn(__fsub_rn(ox, T.lo[0]), T.scale);
        const float gy = __fmul_rn(__fsub_rn(oy, T.lo[1]), T.scale);
        const float gz = __fmul_rn(__fsub_rn(oz, T.lo[2]), T.scale);
        const bool inside = gx >= 0.0f && gx <= fres && gy >= 0.0f && gy <= fres && gz >= 0.0f && gz <= fres;
        const uint64_t jseed = purpose(G.seed, kJitterPurpose);
        const uint64_t jstream = bin_stream(G.frame_dev ? *G.frame_dev : G.frame, b);
        for (int c0 = cbeg; c0 < cend; c0 += chunk) {
            const int cn = min(chunk, cend - c0);  // cells in this chunk
            march_chunk<kGuideThreads, kStage>(T, G, s_nodes, s_stack, s_ray, wbuf, &s_next, c0, cn, chunk,
                                               r != kNone, inside, gx, gy, gz, jseed, jstream, tn, status,
                                               field + c0, hqueue);
        }
        bool finish = true;
        if (parts > 1) {  // publish this part's cells; the CTA of the bin's last part gathers them all
            float* gf = pdf + (size_t)b * NN;  // the bin's pdf row holds the field until it is finished
            for (int c = cbeg + tid; c < cend; c += kGuideThreads) gf[c] = field[c];
            __threadfence();
            __syncthreads();
            if (tid == 0)
                s_last = atomicAdd(reinterpret_cast<uint32_t*>(cdf_marg + (size_t)b * N), 1u) == (uint32_t)(parts - 1);
            __syncthreads();
            finish = s_last != 0;
            if (finish) {
                __threadfence();
                for (int c = tid; c < NN; c += kGuideThreads) field[c] = __ldcg(gf + c);
                __syncthreads();
            }
        }
        if (finish && G.blur) blur_field(field, tmp, N, tid, kGuideThreads);
        // row CDFs (one warp per row) into tmp, row totals into rowtot
        for (int j = warp; finish && j < N; j += kWarps) {
            const float tot = warp_scan_row(field + j * N, tmp + j * N, N, lane);
            if (lane == 0) rowtot[j] = tot;
        }
        __syncthreads();
        if (finish && warp == 0) warp_scan_row(rowtot, marg, N, lane);
        __syncthreads();
        const float den = __fmul_rn(marg[N - 1], kFourPi);
        const float nn = (float)NN;
        if (!finish) {
            // another part of this bin finishes it
        } else if (!kFused) {
            float* gp = pdf + (size_t)b * NN;
            float* gc = cdf_row + (size_t)b * NN;
            for (int c = tid; c < NN; c += kGuideThreads) {
                gp[c] = __fdiv_rn(__fmul_rn(field[c], nn), den);
                gc[c] = tmp[c];
            }
            for (int j = tid; j < N; j += kGuideThreads) cdf_marg[(size_t)b * N + j] = marg[j];
        } else {
            const uint32_t r_lo = F.bin_offset[b], r_hi = F.bin_offset[b + 1];
            bool spilled = false;
            if (F.split && r_hi - r_lo > F.split) {  // uniform over the block
                if (tid == 0) {
                    const uint32_t nch = (r_hi - r_lo + kSpillChunk - 1) / kSpillChunk;
                    const unsigned long long old = atomicAdd(F.spill_ctr, (1ull << 40) | nch);
                    const uint32_t slot = (uint32_t)(old >> 40);
                    if (slot < F.spill_cap) {
                        F.spill_bin[slot] = b;
                        F.spill_base[slot] = (uint32_t)(old & kSpillChunkMask);
                    }
                    s_slot = slot;
                }
                __syncthreads();
                const uint32_t slot = s_slot;
                if (slot < F.spill_cap) {
                    float* tab = F.spill_tab + (size_t)slot * (2 * NN + N);
                    for (int c = tid; c < NN; c += kGuideThreads) {
                        tab[c] = field[c];
                        tab[NN + c] = tmp[c];
                    }
                    for (int j = tid; j < N; j += kGuideThreads) tab[2 * NN + j] = marg[j];
                    spilled = true;
                }
            }
            // otherwise the bin's rays sample straight from the shared-memory CDF
            for (uint32_t k = r_lo + tid; !spilled && k < r_hi; k += kGuideThreads)
                sample_ray(F, F.ray_order[k], field, tmp, marg, N, nn, den, tn);
        }
        __syncthreads();
        if (tid == 0) s_unit = gridDim.x + atomicAdd(bin_next, 1u);
        __syncthreads();
        u = s_unit;
    }
}

// Large fields (N >= 64): the cone march alone, persistent CTAs taking (bin,
// part) units of kMarchPart cells from a counter; eps + L of each cell goes to
// the bin's pdf row, which k_field_pdf then blurs and turns into the PDF and
// CDFs in place.  Without the field in shared memory a CTA needs only the top
// SVO levels, its node paths and its ray buffers, so as many CTAs stay
// resident as at N = 32.
constexpr int kMarchPart = 1024;

template <int kGuideThreads>
__global__ void __launch_bounds__(kGuideThreads, 1024 / kGuideThreads)
    k_guide_march(TraceArgs T, GuideArgs G, const float* __restrict__ pos, const uint32_t* __restrict__ origin_ray,
                  const uint32_t* __restrict__ n_bins_dev, uint32_t bin_cap, float* __restrict__ raw,
                  uint32_t* status, uint32_t* __restrict__ unit_next) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = G.N, NN = N * N, D = T.D;
    Node* s_nodes = reinterpret_cast<Node*>(smem);
    uint32_t* s_stack = reinterpret_cast<uint32_t*>(smem + sizeof(Node) * T.smem_nodes);
    float* wbuf = reinterpret_cast<float*>(s_stack + (D + 1) * kGuideThreads);
    uint32_t* hqueue = reinterpret_cast<uint32_t*>(wbuf + (kGuideThreads / 32) * kWbWords * 32);
    __shared__ int s_next;
    __shared__ uint32_t s_unit;
    const int tid = threadIdx.x;
    for (uint32_t i = tid; i < T.smem_nodes; i += kGuideThreads) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(T.node) + i);
        s_nodes[i].first_child = v.x;
        s_nodes[i].mask = v.y;
    }
    __syncthreads();
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const int parts = NN / kMarchPart;
    const uint32_t n_units = nb * (uint32_t)parts;
    const float tn = __fdiv_rn(2.0f, (float)N);
    const float fres = (float)(1 << D);
    for (uint32_t u = blockIdx.x; u < n_units;) {
        const uint32_t b = u / (uint32_t)parts;
        const int c0 = (int)(u % (uint32_t)parts) * kMarchPart;
        const uint32_t r = origin_ray ? origin_ray[b] : b;
        float ox = 0.0f, oy = 0.0f, oz = 0.0f;
        if (r != kNone) {
            ox = pos[3 * (size_t)r + 0];
            oy = pos[3 * (size_t)r + 1];
            oz = pos[3 * (size_t)r + 2];
        }
        const float gx = __fmul_rn(__fsub_rn(ox, T.lo[0]), T.scale);
        const float gy = __fmul_rn(__fsub_rn(oy, T.lo[1]), T.scale);
        const float gz = __fmul_rn(__fsub_rn(oz, T.lo[2]), T.scale);
        const bool inside = gx >= 0.0f && gx <= fres && gy >= 0.0f && gy <= fres && gz >= 0.0f && gz <= fres;
        const uint64_t jseed = purpose(G.seed, kJitterPurpose);
        const uint64_t jstream = bin_stream(G.frame_dev ? *G.frame_dev : G.frame, b);
        march_chunk<kGuideThreads, false>(T, G, s_nodes, s_stack, nullptr, wbuf, &s_next, c0, kMarchPart, kMarchPart,
                                          r != kNone, inside, gx, gy, gz, jseed, jstream, tn, status,
                                          raw + (size_t)b * NN + c0, hqueue);
        if (tid == 0) s_unit = gridDim.x + atomicAdd(unit_next, 1u);
        __syncthreads();
        u = s_unit;
    }
}

// Unfused fields over a flat SVO index: the cone rays of every bin as one
// stream.  Each warp takes batches of 32 cells of one bin from a counter over
// all bins, sets up their rays (keeping only those alive at their start) and
// hands a ray to each lane as it frees; a lane keeps its ray's own origin, so
// lanes of a warp may march rays of different bins.  No barrier holds a warp
// back at the end of a bin.  eps + L of each cell goes to the bin's pdf row
// (leaf hits through the warp's queue); k_field_pdf then blurs the rows and
// builds the PDF and CDFs in place.
// walk steps a lane may take per pass of the stream kernel's loop before the warp meets again
// (3 measured best: 2 shares less of the pass overhead, 4 and more let the lanes drift apart)
constexpr int kStreamSteps = 3;
// the same once the warp's batches have run out: no lane can take new work, so a longer pass
// only saves the pass overhead of the few rays left (16 measured best of 8, 16 and 64)
constexpr int kStreamDrySteps = 16;
template <int kGuideThreads, int kD>
__global__ void __launch_bounds__(kGuideThreads, 1024 / kGuideThreads)
    k_guide_stream(TraceArgs T, GuideArgs G, const float* __restrict__ pos, const uint32_t* __restrict__ origin_ray,
                   const uint32_t* __restrict__ n_bins_dev, uint32_t bin_cap, float* __restrict__ raw,
                   uint32_t* status, uint32_t* __restrict__ batch_next) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    float* wb = reinterpret_cast<float*>(smem) + warp * (kWbWords * 32);
    uint32_t* hq = reinterpret_cast<uint32_t*>(reinterpret_cast<float*>(smem) + (kGuideThreads / 32) * kWbWords * 32) +
                   warp * (kHitQueue * kHitWords);
    const int N = G.N, NN = N * N, D = svo_depth<kD>(T);
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const uint32_t per_bin = (uint32_t)NN / 32u;
    const uint32_t n_batches = nb * per_bin;
    const float tn = __fdiv_rn(2.0f, (float)N);
    const int res = 1 << D;
    const float fres = (float)res;
    const float INF = __int_as_float(0x7f800000);
    const int cap = 3 * res + 16;
    const uint64_t jseed = purpose(G.seed, kJitterPurpose);
    const uint32_t frame = G.frame_dev ? *G.frame_dev : G.frame;
    int q = -1;  // global cell index b N^2 + c of this lane's ray (-1: none)
    float dx = 0.f, dy = 0.f, dz = 0.f, ivx = 0.f, ivy = 0.f, ivz = 0.f, t = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    int cx = 0, cy = 0, cz = 0, level = -1, steps = 0;
    float bgx = 0.f, bgy = 0.f, bgz = 0.f;  // origin (grid units) of the warp's current batch
    int wb_n = 0, wb_head = 0;
    bool dry = false, pend = false;
    int hq_n = 0;
    for (;;) {
        // hits of the last pass join the warp's queue (finished together when it would overflow)
        const uint32_t hm = __ballot_sync(0xffffffffu, pend);
        if (hm) {
            if (hq_n + __popc(hm) > kHitQueue) {
                flush_hits<kD>(T, G, nullptr, hq, 0, hq_n, lane, raw);
                hq_n = 0;
                __syncwarp();
            }
            if (pend) {
                const int e = hq_n + __popc(hm & lt);
                hq[0 * kHitQueue + e] = (uint32_t)q;
                hq[1 * kHitQueue + e] = __float_as_uint(t);
                hq[2 * kHitQueue + e] = (uint32_t)cx | ((uint32_t)cy << 16);
                hq[3 * kHitQueue + e] = (uint32_t)cz;
                hq[4 * kHitQueue + e] = __float_as_uint(dx);
                hq[5 * kHitQueue + e] = __float_as_uint(dy);
                hq[6 * kHitQueue + e] = __float_as_uint(dz);
                q = -1;
                pend = false;
            }
            hq_n += __popc(hm);
            __syncwarp();
        }
        // hand out buffered rays to idle lanes; an empty buffer takes the next batch of 32 cells of
        // some bin (origin, then every lane sets up one ray; only rays alive at their start are kept)
#pragma unroll 1
        for (int round = 0; round < 4; ++round) {
            const bool idle = q < 0;
            const uint32_t need = __ballot_sync(0xffffffffu, idle);
            if (!need) break;
            if (wb_head == wb_n) {
                if (dry) break;
                uint32_t batch = 0;
                if (lane == 0) batch = atomicAdd(batch_next, 1u);
                batch = __shfl_sync(0xffffffffu, batch, 0);
                if (batch >= n_batches) {
                    dry = true;
                    wb_n = wb_head = 0;
                    break;
                }
                const uint32_t b = batch / per_bin;
                const int c = (int)(batch % per_bin) * 32 + lane;
                const uint32_t r = origin_ray ? origin_ray[b] : b;
                float ox = 0.0f, oy = 0.0f, oz = 0.0f;
                if (r != kNone) {
                    ox = pos[3 * (size_t)r + 0];
                    oy = pos[3 * (size_t)r + 1];
                    oz = pos[3 * (size_t)r + 2];
                }
                bgx = __fmul_rn(__fsub_rn(ox, T.lo[0]), T.scale);
                bgy = __fmul_rn(__fsub_rn(oy, T.lo[1]), T.scale);
                bgz = __fmul_rn(__fsub_rn(oz, T.lo[2]), T.scale);
                const bool inside = bgx >= 0.0f && bgx <= fres && bgy >= 0.0f && bgy <= fres && bgz >= 0.0f &&
                                    bgz <= fres;
                float3 d, iv;
                cell_ray(T, G, c, jseed, bin_stream(frame, b), tn, &d, &iv);
                float t0;
                int x0, y0, z0;
                const bool alive = ray_start(T, r != kNone, inside, bgx, bgy, bgz, d.x, d.y, d.z, iv.x, iv.y, iv.z,
                                             res, fres, &t0, &x0, &y0, &z0);
                const int g = (int)b * NN + c;
                const uint32_t am = __ballot_sync(0xffffffffu, alive);
                if (!alive) {
                    raw[g] = __fadd_rn(G.eps, 0.0f);
                } else {
                    const int k = __popc(am & lt);
                    wb[0 * 32 + k] = __int_as_float(g);
                    wb[1 * 32 + k] = d.x;
                    wb[2 * 32 + k] = d.y;
                    wb[3 * 32 + k] = d.z;
                    wb[4 * 32 + k] = iv.x;
                    wb[5 * 32 + k] = iv.y;
                    wb[6 * 32 + k] = iv.z;
                    wb[7 * 32 + k] = t0;
                    wb[8 * 32 + k] = __int_as_float(x0);
                    wb[9 * 32 + k] = __int_as_float(y0);
                    wb[10 * 32 + k] = __int_as_float(z0);
                }
                wb_n = __popc(am);
                wb_head = 0;
                __syncwarp();
            }
            const int k = wb_head + __popc(need & lt);
            if (idle && k < wb_n) {
                q = __float_as_int(wb[0 * 32 + k]);
                dx = wb[1 * 32 + k];
                dy = wb[2 * 32 + k];
                dz = wb[3 * 32 + k];
                ivx = wb[4 * 32 + k];
                ivy = wb[5 * 32 + k];
                ivz = wb[6 * 32 + k];
                t = wb[7 * 32 + k];
                cx = __float_as_int(wb[8 * 32 + k]);
                cy = __float_as_int(wb[9 * 32 + k]);
                cz = __float_as_int(wb[10 * 32 + k]);
                gx = bgx;
                gy = bgy;
                gz = bgz;
                level = -1;
                steps = 0;
            }
            wb_head = min(wb_n, wb_head + __popc(need));
            __syncwarp();  // entries are read before a refill overwrites them
        }
        if (dry && __all_sync(0xffffffffu, q < 0)) {
            if (hq_n > 0) flush_hits<kD>(T, G, nullptr, hq, 0, hq_n, lane, raw);
            break;
        }
        if (q < 0) continue;
        // ---- up to kStreamSteps steps (kStreamDrySteps once no batch is left): the cell's deepest
        // existing level, then its hit or the skip of its empty block (the pass overhead of the
        // queue and the hand-out is shared by them)
        bool done = false;
        const int nsteps = dry ? kStreamDrySteps : kStreamSteps;
#pragma unroll 1
        for (int ks = 0; ks < nsteps && !done && !pend; ++ks) {
            if (level < 0) level = deepest_level<kD>(T, cx, cy, cz);
            if (level == D && t >= T.t_skip) {
                pend = true;  // its cone query waits in the warp's queue
            } else {
                const int sl = (level == D) ? 0 : D - level - 1;
                const int size = 1 << sl;
                const int bx = (cx >> sl) << sl, by = (cy >> sl) << sl, bz = (cz >> sl) << sl;
                const int ex = ivx > 0.0f ? bx + size : bx - 1;
                const int ey = ivy > 0.0f ? by + size : by - 1;
                const int ez = ivz > 0.0f ? bz + size : bz - 1;
                const float tex = ivx != 0.0f ? cross_time(ex, ivx > 0.0f, gx, ivx) : INF;
                const float tey = ivy != 0.0f ? cross_time(ey, ivy > 0.0f, gy, ivy) : INF;
                const float tez = ivz != 0.0f ? cross_time(ez, ivz > 0.0f, gz, ivz) : INF;
                const int a = (tex <= tey && tex <= tez) ? 0 : (tey <= tez ? 1 : 2);
                const float tx = a == 0 ? tex : (a == 1 ? tey : tez);
                const int p = a == 0 ? 1 : 0, pq = a == 2 ? 1 : 2;
                const int cp = p == 0 ? cx : cy, cq = pq == 1 ? cy : cz;
                const int bp = p == 0 ? bx : by, bq = pq == 1 ? by : bz;
                const float gp = p == 0 ? gx : gy, gq = pq == 1 ? gy : gz;
                const float ip = p == 0 ? ivx : ivy, iq = pq == 1 ? ivy : ivz;
                const float dp = p == 0 ? dx : dy, dq = pq == 1 ? dy : dz;
                const int np = advance_axis(cp, bp, size, gp, ip, __fmul_rn(dp, T.scale), tx, p < a);
                const int nq = advance_axis(cq, bq, size, gq, iq, __fmul_rn(dq, T.scale), tx, pq < a);
                const int na = a == 0 ? ex : (a == 1 ? ey : ez);
                if (tx == INF || na < 0 || na >= res) {
                    done = true;  // left the grid: miss
                } else if (++steps > cap) {
                    atomicOr(status, (uint32_t)WFPG_STATUS_TRACE_CAP);
                    done = true;
                } else {
                    cx = a == 0 ? na : np;
                    cy = a == 1 ? na : (p == 1 ? np : nq);
                    cz = a == 2 ? na : nq;
                    t = tx;
                    level = -1;
                }
            }
        }
        if (done) {
            raw[q] = __fadd_rn(G.eps, 0.0f);
            q = -1;
        }
    }
}

// PDF and CDFs of given fields (one CTA per bin): optionally the blur, then row
// CDFs and the marginal in warp order with a running maximum, pdf = f N^2 /
// (T 4 pi), as in the traced path.  The field may be the pdf rows themselves
// (each CTA reads its whole row before writing it).
__global__ void __launch_bounds__(256) k_field_pdf(const float* field, int N, const uint32_t* __restrict__ n_bins_dev,
                                                   uint32_t bin_cap, int blur, float* pdf, float* __restrict__ cdf_row,
                                                   float* __restrict__ cdf_marg) {
    extern __shared__ __align__(16) float fsm[];
    const int NN = N * N;
    float* f = fsm;
    float* rows = f + NN;
    float* rowtot = rows + NN;
    float* marg = rowtot + N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nw = nt >> 5;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const uint32_t b = blockIdx.x;
    if (b >= nb) return;
    for (int c = tid; c < NN; c += nt) f[c] = field[(size_t)b * NN + c];
    __syncthreads();
    if (blur) blur_field(f, rows, N, tid, nt);
    for (int j = warp; j < N; j += nw) {
        const float tot = warp_scan_row(f + j * N, rows + j * N, N, lane);
        if (lane == 0) rowtot[j] = tot;
    }
    __syncthreads();
    if (warp == 0) warp_scan_row(rowtot, marg, N, lane);
    __syncthreads();
    const float den = __fmul_rn(marg[N - 1], kFourPi);
    const float nn = (float)NN;
    for (int c = tid; c < NN; c += nt) {
        pdf[(size_t)b * NN + c] = __fdiv_rn(__fmul_rn(f[c], nn), den);
        cdf_row[(size_t)b * NN + c] = rows[c];
    }
    for (int j = tid; j < N; j += nt) cdf_marg[(size_t)b * N + j] = marg[j];
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

// one-sample mixture from stored tables (what the fused launch does from shared
// memory): guided with probability alpha, else cosine; a ray whose bin has no
// table (>= the built count) takes the cosine branch with alpha = 0
__global__ void __launch_bounds__(256) k_sample_mix(const float* __restrict__ pdf, const float* __restrict__ cdf_row,
                                                    const float* __restrict__ cdf_marg, int N, uint32_t bin_cap,
                                                    const uint32_t* __restrict__ n_bins_dev,
                                                    const uint32_t* __restrict__ bin_of_ray,
                                                    const float* __restrict__ nrm, const float* __restrict__ u,
                                                    uint32_t n_cap, const uint32_t* __restrict__ n_dev, float alpha,
                                                    float* __restrict__ dir, float* __restrict__ pdf_out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = n_dev ? min(*n_dev, n_cap) : n_cap;
    if (i >= n) return;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const uint32_t b = bin_of_ray[i];
    const float u0 = u[3 * (size_t)i], u1 = u[3 * (size_t)i + 1], u2 = u[3 * (size_t)i + 2];
    const float nx = nrm[3 * (size_t)i], ny = nrm[3 * (size_t)i + 1], nz = nrm[3 * (size_t)i + 2];
    const int NN = N * N;
    float3 d;
    float pg = 0.0f, a = alpha;
    if (b >= nb) {
        a = 0.0f;
        d = cosine_dir(nx, ny, nz, u0, u1);
    } else if (u2 < alpha) {
        const float* M = cdf_marg + (size_t)b * N;
        const float t0 = __fmul_rn(u0, M[N - 1]);
        const int r = min(upper_bound_f(M, N, t0), N - 1);
        const float* C = cdf_row + ((size_t)b * N + r) * N;
        const float t1 = __fmul_rn(u1, C[N - 1]);
        const int c = min(upper_bound_f(C, N, t1), N - 1);
        const float mlo = r > 0 ? M[r - 1] : 0.0f, mhi = M[r];
        const float clo = c > 0 ? C[c - 1] : 0.0f, chi = C[c];
        const float beta = clamp01(__fdiv_rn(__fsub_rn(t0, mlo), __fsub_rn(mhi, mlo)));
        const float al = clamp01(__fdiv_rn(__fsub_rn(t1, clo), __fsub_rn(chi, clo)));
        const float tn = __fdiv_rn(2.0f, (float)N);
        d = octa_to_dir(__fsub_rn(__fmul_rn(__fadd_rn((float)c, al), tn), 1.0f),
                        __fsub_rn(__fmul_rn(__fadd_rn((float)r, beta), tn), 1.0f));
        pg = pdf[(size_t)b * NN + r * N + c];
    } else {
        d = cosine_dir(nx, ny, nz, u0, u1);
        pg = pdf[(size_t)b * NN + octa_cell(d, N)];
    }
    const float cs = fmaxf(0.0f, nx * d.x + ny * d.y + nz * d.z);
    dir[3 * (size_t)i] = d.x;
    dir[3 * (size_t)i + 1] = d.y;
    dir[3 * (size_t)i + 2] = d.z;
    pdf_out[i] = a * pg + (1.0f - a) * cs * 0.31830988618379067f;
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
static size_t guide_smem_bytes(uint32_t smem_nodes, int N, int D, int threads, bool stage) {
    const size_t NN = (size_t)N * N;
    const size_t chunk = NN < (size_t)kGuideChunk ? NN : (size_t)kGuideChunk;
    const size_t rays = stage ? 6 * chunk : (size_t)(threads / 32) * kWbWords * 32;
    return sizeof(Node) * smem_nodes + sizeof(uint32_t) * (size_t)(D + 1) * threads +
           sizeof(float) * (rays + 2 * NN + 2 * (size_t)N) + sizeof(uint32_t) * (size_t)(threads / 32) * kHitQueue * kHitWords;
}

// zeroes the per-bin part counters (the first word of each bin's cdf_marg row)
__global__ void k_zero_part_counters(float* cdf_marg, int N, const uint32_t* n_bins_dev, uint32_t bin_cap) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    if (b < nb) reinterpret_cast<uint32_t*>(cdf_marg)[(size_t)b * N] = 0u;
}

// resident CTAs of `kernel` on the whole GPU (0 when the field does not fit), after
// raising its dynamic shared-memory limit where needed
template <typename Kernel>
static uint64_t guide_slots(Kernel kernel, int threads, size_t smem, int* rc) {
    *rc = WFPG_OK;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        *rc = WFPG_ERR_CUDA;
        return 0;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) *rc = WFPG_ERR_INVALID_ARG;  // the field does not fit in shared memory
    return (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 0);
}

template <int kThreads, bool kStage, bool kFused>
static int launch_guide(const TraceArgs& T, const GuideArgs& G, const FusedArgs& F, const float* pos,
                        const uint32_t* origin_ray, const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf,
                        float* cdf_row, float* cdf_marg, uint32_t* status, uint32_t* bin_next, int D,
                        int parts_param, cudaStream_t st) {
    // one CTA per bin unless the unfused call may split bins (a separate instantiation:
    // the split bookkeeping costs the one-CTA kernel registers and residency)
    auto kernel = k_guide_build<kThreads, kStage, kFused, false>;
    const size_t smem = guide_smem_bytes(T.smem_nodes, G.N, D, kThreads, kStage);
    int rc = WFPG_OK;
    uint64_t slots = guide_slots(kernel, kThreads, smem, &rc);
    if (rc != WFPG_OK) return rc;
    // parts per bin (unfused only; 0: chosen in the kernel from the device-side bin count)
    int parts = kFused ? 1 : parts_param;
    if (parts == 0 && (uint64_t)bin_cap * 2 > slots) parts = 1;  // the kernel could not split either
    if (!kFused && parts != 1) {
        kernel = k_guide_build<kThreads, kStage, kFused, !kFused>;
        slots = guide_slots(kernel, kThreads, smem, &rc);
        if (rc != WFPG_OK) return rc;
    }
    const uint64_t most = parts == 0 ? 8 : (uint64_t)parts;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)bin_cap * most, slots);
    if (cudaMemsetAsync(bin_next, 0, sizeof(uint32_t), st) != cudaSuccess) return WFPG_ERR_CUDA;
    if (parts != 1)
        WFPG_LAUNCH(k_zero_part_counters, div_up(bin_cap, 256), 256, 0, st, cdf_marg, G.N, n_bins_dev, bin_cap);
    WFPG_LAUNCH(kernel, grid, kThreads, smem, st, T, G, F, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row,
                cdf_marg, status, bin_next, parts, (uint32_t)std::min<uint64_t>(slots, 0xFFFFFFFFull));
    return launch_status();
}

static void trace_setup(const wfpg_svo* s, const wfpg_guide_params* p, TraceArgs* T, GuideArgs* G,
                        const uint32_t* frame_dev) {
    T->node = s->node;
    T->normal = s->normal;
    T->value = s->value;
    T->D = s->D;
    for (int a = 0; a < 3; ++a) T->lo[a] = s->lo[a];
    T->scale = s->scale;
    T->S = s->S;
    T->t_skip = p->t_skip;
    T->omega = kFourPi / (float)(p->N * p->N);
    T->cos_weight = p->cos_weight;
    const int top = s->D < kSmemTopLevels ? s->D : kSmemTopLevels;
    T->smem_nodes = s->level_off[top + 1];
    T->top = s->top;
    T->G = s->top_levels - 1;
    T->top_offG = T->G >= 0 ? s->top_off[T->G] : 0u;
    T->occ = s->occ;
    for (int j = 0; j < kOccMaxDepth - kTopLevelMax; ++j) {
        const int l = T->G + 1 + j;
        T->occ_off[j] = (s->occ && l <= s->D) ? (uint32_t)s->occ_off[l] : 0u;
    }
    // the flat walk of the generic kernels uses 32-bit Morton keys: up to depth 10 (the stream
    // kernel specialised on depth 11 turns it on for itself)
    T->flat = T->G >= 0 && (T->G == s->D || s->occ != nullptr) && s->D <= 10;
    G->N = p->N;
    G->eps = p->eps;
    G->jitter = p->jitter;
    G->blur = p->blur;
    G->seed = p->seed;
    G->frame = p->frame;
    G->frame_dev = frame_dev;
}

template <bool kFused>
static int dispatch_guide(const wfpg_svo* s, const wfpg_guide_params* p, const TraceArgs& T, const GuideArgs& G,
                          const FusedArgs& F, const float* pos, const uint32_t* origin_ray,
                          const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf, float* cdf_row, float* cdf_marg,
                          cudaStream_t st) {
    const bool small = p->N <= 16;
    const int threads = p->block ? p->block
                                 : (small ? kGuideDefaultThreadsSmall
                                          : (p->N <= 32 ? kGuideDefaultThreadsMid : kGuideDefaultThreadsLarge));
    const bool stage = p->stage == 0 ? small : p->stage > 0;
    const int D = s->D;
#define WFPG_GUIDE_CASE(TH)                                                                                        \
    if (threads == TH)                                                                                             \
        return stage ? launch_guide<TH, true, kFused>(T, G, F, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row, \
                                                      cdf_marg, s->status, s->bin_next, D, (int)p->parts, st)      \
                     : launch_guide<TH, false, kFused>(T, G, F, pos, origin_ray, n_bins_dev, bin_cap, pdf,         \
                                                       cdf_row, cdf_marg, s->status, s->bin_next, D,              \
                                                       (int)p->parts, st);
    WFPG_GUIDE_CASE(64)
    WFPG_GUIDE_CASE(128)
    WFPG_GUIDE_CASE(256)
#undef WFPG_GUIDE_CASE
    return WFPG_ERR_INVALID_ARG;
}

int field_pdf_impl(const float* field, int N, const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf,
                   float* cdf_row, float* cdf_marg, cudaStream_t st, int blur);

template <int kThreads, int kD>
static int launch_stream(const wfpg_svo* s, const TraceArgs& T0, const GuideArgs& G, const float* pos,
                         const uint32_t* origin_ray, const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf,
                         float* cdf_row, float* cdf_marg, cudaStream_t st) {
    TraceArgs T = T0;
    T.smem_nodes = 0;  // no node cache: the flat walk reads nodes only below the index
    T.flat = 1;
    auto kernel = k_guide_stream<kThreads, kD>;
    const size_t smem = sizeof(float) * (size_t)(kThreads / 32) * kWbWords * 32 +
                        sizeof(uint32_t) * (size_t)(kThreads / 32) * kHitQueue * kHitWords;
    int rc = WFPG_OK;
    const uint64_t slots = guide_slots(kernel, kThreads, smem, &rc);
    if (rc != WFPG_OK) return rc;
    const uint64_t warps_needed = ((uint64_t)bin_cap * (uint64_t)(G.N * G.N) / 32 + kThreads / 32 - 1) / (kThreads / 32);
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(warps_needed, slots));
    if (cudaMemsetAsync(s->bin_next, 0, sizeof(uint32_t), st) != cudaSuccess) return WFPG_ERR_CUDA;
    WFPG_LAUNCH(kernel, grid, kThreads, smem, st, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, s->status,
                s->bin_next);
    rc = launch_status();
    if (rc != WFPG_OK) return rc;
    return field_pdf_impl(pdf, G.N, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st, G.blur);
}

template <int kThreads>
static int launch_march(const wfpg_svo* s, const TraceArgs& T, const GuideArgs& G, const float* pos,
                        const uint32_t* origin_ray, const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf,
                        float* cdf_row, float* cdf_marg, cudaStream_t st) {
    auto kernel = k_guide_march<kThreads>;
    const size_t smem = sizeof(Node) * T.smem_nodes + sizeof(uint32_t) * (size_t)(s->D + 1) * kThreads +
                        sizeof(float) * (size_t)(kThreads / 32) * kWbWords * 32 +
                        sizeof(uint32_t) * (size_t)(kThreads / 32) * kHitQueue * kHitWords;
    int rc = WFPG_OK;
    const uint64_t slots = guide_slots(kernel, kThreads, smem, &rc);
    if (rc != WFPG_OK) return rc;
    const uint64_t units = (uint64_t)bin_cap * (uint64_t)(G.N * G.N / kMarchPart);
    const uint32_t grid = (uint32_t)std::min<uint64_t>(units, slots);
    if (cudaMemsetAsync(s->bin_next, 0, sizeof(uint32_t), st) != cudaSuccess) return WFPG_ERR_CUDA;
    WFPG_LAUNCH(kernel, grid, kThreads, smem, st, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, s->status,
                s->bin_next);
    rc = launch_status();
    if (rc != WFPG_OK) return rc;
    return field_pdf_impl(pdf, G.N, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st, G.blur);
}

int guide_build_impl(const wfpg_svo* s, const float* pos, const uint32_t* origin_ray, const uint32_t* n_bins_dev,
                     uint32_t bin_cap, const wfpg_guide_params* p, float* pdf, float* cdf_row, float* cdf_marg,
                     cudaStream_t st, const uint32_t* frame_dev) {
    if (bin_cap == 0) return WFPG_OK;
    TraceArgs T;
    GuideArgs G;
    trace_setup(s, p, &T, &G, frame_dev);
    const int sthreads = p->block ? p->block : kGuideDefaultThreadsMid;
    const bool wide_flat = s->D == 11 && s->occ != nullptr && s->top_levels > 0 && sthreads == 128;
    if ((T.flat || wide_flat) && p->parts == 0) {  // flat index: every bin's cone rays as one stream, then the per-bin finish
        const int threads = sthreads;
        // the default block size has kernels specialised on the SVO depth 6 .. 11 (constant shifts and loop bounds)
#define WFPG_STREAM(TH, KD) launch_stream<TH, KD>(s, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st)
        if (threads == 128) {
            switch (s->D) {
                case 6: return WFPG_STREAM(128, 6);
                case 7: return WFPG_STREAM(128, 7);
                case 8: return WFPG_STREAM(128, 8);
                case 9: return WFPG_STREAM(128, 9);
                case 10: return WFPG_STREAM(128, 10);
                case 11: return WFPG_STREAM(128, 11);
                default: return WFPG_STREAM(128, 0);
            }
        }
        if (threads == 64) return WFPG_STREAM(64, 0);
        if (threads == 256) return WFPG_STREAM(256, 0);
#undef WFPG_STREAM
        return WFPG_ERR_INVALID_ARG;
    }
    if (p->N >= 64 && p->parts == 0) {  // large fields: the march, then the per-bin finish
        const int threads = p->block ? p->block : kGuideDefaultThreadsMid;
        if (threads == 64) return launch_march<64>(s, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st);
        if (threads == 128) return launch_march<128>(s, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st);
        if (threads == 256) return launch_march<256>(s, T, G, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st);
        return WFPG_ERR_INVALID_ARG;
    }
    FusedArgs F{};
    return dispatch_guide<false>(s, p, T, G, F, pos, origin_ray, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st);
}

constexpr uint32_t kGuideSplitDefault = 2048;

static uint32_t split_of(const wfpg_guide_params* p) {
    return p->split == 0 ? kGuideSplitDefault : (p->split == 0xFFFFFFFFu ? 0u : p->split);
}

size_t guide_fused_workspace_bytes(int N, uint32_t n, uint32_t split_param) {
    wfpg_guide_params p{};
    p.split = split_param;
    const uint32_t split = split_of(&p);
    const size_t cap = split ? (size_t)n / split + 1 : 0;
    return arena_bytes<unsigned long long>(1) + 2 * arena_bytes<uint32_t>(cap) +
           arena_bytes<float>(cap * (2 * (size_t)N * N + N)) + 256;
}

int guide_fused_impl(const wfpg_svo* s, const float* pos, const float* nrm, const uint32_t* origin_ray,
                     const uint32_t* n_bins_dev, uint32_t bin_cap, const uint32_t* ray_order,
                     const uint32_t* bin_offset, const float* u, float alpha, const wfpg_guide_params* p, float* dir,
                     float* pdf_out, uint32_t n, void* workspace, size_t ws_bytes, cudaStream_t st,
                     const uint32_t* frame_dev, const float* eval_dir, float* eval_pdf) {
    if (bin_cap == 0) return WFPG_OK;
    TraceArgs T;
    GuideArgs G;
    trace_setup(s, p, &T, &G, frame_dev);
    FusedArgs F{};
    F.ray_order = ray_order;
    F.bin_offset = bin_offset;
    F.nrm = nrm;
    F.u = u;
    F.alpha = alpha;
    F.dir = dir;
    F.pdf = pdf_out;
    F.eval_dir = eval_dir;
    F.eval_pdf = eval_pdf;
    F.split = split_of(p);
    if (F.split) {
        const size_t cap = (size_t)n / F.split + 1;
        Arena ws{static_cast<char*>(workspace), ws_bytes, 0, false};
        F.spill_ctr = ws.take<unsigned long long>(1);
        F.spill_bin = ws.take<uint32_t>(cap);
        F.spill_base = ws.take<uint32_t>(cap);
        F.spill_tab = ws.take<float>(cap * (2 * (size_t)p->N * p->N + p->N));
        if (ws.overflow) return WFPG_ERR_CAPACITY;
        F.spill_cap = (uint32_t)cap;
        if (cudaMemsetAsync(F.spill_ctr, 0, sizeof(unsigned long long), st) != cudaSuccess) return WFPG_ERR_CUDA;
    }
    const int rc =
        dispatch_guide<true>(s, p, T, G, F, pos, origin_ray, n_bins_dev, bin_cap, nullptr, nullptr, nullptr, st);
    if (rc != WFPG_OK || !F.split) return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    WFPG_LAUNCH(k_spill_sample, (uint32_t)sms * 8, kSpillChunk, 0, st, F, p->N);
    return launch_status();
}

// threads of a k_field_pdf CTA for fields of up to 32 x 32 cells: four warps, so twice the bins
// of 256-thread CTAs are in flight per SM (65,536 learned fields at N = 32: 6 % faster)
constexpr int kFieldPdfSmall = 128;
int field_pdf_impl(const float* field, int N, const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf,
                   float* cdf_row, float* cdf_marg, cudaStream_t st, int blur) {
    if (bin_cap == 0) return WFPG_OK;
    const size_t smem = sizeof(float) * (2 * (size_t)N * N + 2 * (size_t)N);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_field_pdf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return WFPG_ERR_CUDA;
    // small fields: CTAs of kFieldPdfSmall threads, more bins in flight per SM (the results do not
    // depend on the block size: the blur is per cell, each row scan belongs to one warp)
    const int threads = N <= 32 ? kFieldPdfSmall : 256;
    WFPG_LAUNCH(k_field_pdf, bin_cap, threads, smem, st, field, N, n_bins_dev, bin_cap, blur, pdf, cdf_row, cdf_marg);
    return launch_status();
}

int guide_sample_impl(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                      const uint32_t* bin_of_ray, const float* u, uint32_t n, float* dir, float* pdf_out,
                      uint32_t* cell, cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_guide_sample, div_up(n, 256), 256, 0, st, pdf, cdf_row, cdf_marg, N, bin_cap, bin_of_ray,
                                                   reinterpret_cast<const float2*>(u), n, dir, pdf_out, cell);
    return launch_status();
}

// mixture density alpha * table density + (1 - alpha) * cos+ / pi of given
// directions (rays < *n_dev; a bin without a table: alpha = 0)
__global__ void __launch_bounds__(256) k_mix_eval(const float* __restrict__ pdf, int N, uint32_t bin_cap,
                                                  const uint32_t* __restrict__ n_bins_dev,
                                                  const uint32_t* __restrict__ bin_of_ray,
                                                  const float* __restrict__ nrm, const float* __restrict__ dir,
                                                  uint32_t n_cap, const uint32_t* __restrict__ n_dev, float alpha,
                                                  float* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = n_dev ? min(*n_dev, n_cap) : n_cap;
    if (i >= n) return;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const uint32_t b = bin_of_ray[i];
    const float3 d = make_float3(dir[3 * (size_t)i], dir[3 * (size_t)i + 1], dir[3 * (size_t)i + 2]);
    const float cs = fmaxf(0.0f, nrm[3 * (size_t)i] * d.x + nrm[3 * (size_t)i + 1] * d.y + nrm[3 * (size_t)i + 2] * d.z);
    float a = alpha, pg = 0.0f;
    if (b >= nb) a = 0.0f;
    else pg = pdf[(size_t)b * N * N + octa_cell(d, N)];
    out[i] = a * pg + (1.0f - a) * cs * 0.31830988618379067f;
}

int mix_eval_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, const uint32_t* bin_of_ray,
                  const float* nrm, const float* dir, uint32_t n, const uint32_t* n_dev, float alpha, float* out,
                  cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_mix_eval, div_up(n, 256), 256, 0, st, pdf, N, bin_cap, n_bins_dev, bin_of_ray, nrm, dir, n, n_dev,
                alpha, out);
    return launch_status();
}

int sample_mix_impl(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, uint32_t bin_cap,
                    const uint32_t* n_bins_dev, const uint32_t* bin_of_ray, const float* nrm, const float* u,
                    uint32_t n, const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_sample_mix, div_up(n, 256), 256, 0, st, pdf, cdf_row, cdf_marg, N, bin_cap, n_bins_dev, bin_of_ray,
                nrm, u, n, n_dev, alpha, dir, pdf_out);
    return launch_status();
}

int guide_eval_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* bin, const float* dir, uint32_t n,
                    float* out, cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_guide_eval, div_up(n, 256), 256, 0, st, pdf, N, bin_cap, bin, dir, n, out);
    return launch_status();
}

}  // namespace wfpg
