// UpdateExitance (Alg. 1, Eq. 5) and the bottom-up average (Sec. 3.2).
//
// Records are scattered with unsigned 64-bit fixed-point atomics (2^-20
// units), so the cached sums do not depend on the order the records arrive
// in; the average is then rebuilt level by level from the leaves up, each
// child side routed to the parent side its normal agrees with.
#include "common.cuh"
#include "svo.cuh"

namespace wfpg {

struct AccArgs {  // the tree and the grid mapping the scatter needs
    const Node* node;
    const float4* normal;
    int D;
    float lo[3];
    float scale;
};

__global__ void __launch_bounds__(256) k_accumulate(AccArgs A, const float* __restrict__ pos,
                                                    const float* __restrict__ wout, const float* __restrict__ L,
                                                    uint32_t n, const uint32_t* __restrict__ n_dev,
                                                    unsigned long long* __restrict__ acc_sum,
                                                    uint32_t* __restrict__ acc_cnt) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (n_dev ? min(*n_dev, n) : n)) return;
    int c[3];
    c[0] = grid_index(pos[3 * (size_t)i + 0], A.lo[0], A.scale, A.D);
    c[1] = grid_index(pos[3 * (size_t)i + 1], A.lo[1], A.scale, A.D);
    c[2] = grid_index(pos[3 * (size_t)i + 2], A.lo[2], A.scale, A.D);
    int lvl;
    const uint32_t nd = descend(A.node, c, A.D, &lvl);
    const float4 N = A.normal[nd];
    const float wx = wout[3 * (size_t)i + 0], wy = wout[3 * (size_t)i + 1], wz = wout[3 * (size_t)i + 2];
    const float d = __fadd_rn(__fadd_rn(__fmul_rn(N.x, wx), __fmul_rn(N.y, wy)), __fmul_rn(N.z, wz));
    const int side = (d >= 0.0f) ? 0 : 1;
    const float Li = L[i];
    const float Lc = (Li > 0.0f) ? fminf(Li, 16777216.0f) : 0.0f;
    const unsigned long long q = __float2ull_rn(__fmul_rn(Lc, 1048576.0f));
    atomicAdd(&acc_sum[2 * (size_t)nd + side], q);
    atomicAdd(&acc_cnt[2 * (size_t)nd + side], 1u);
}

__device__ __forceinline__ float side_value(unsigned long long sum, uint32_t cnt) {
    return __fdiv_rn(__fmul_rn(__ull2float_rn(sum), 0x1p-20f), __uint2float_rn(cnt));
}
__device__ __forceinline__ float2 node_values(unsigned long long s0, uint32_t c0, unsigned long long s1, uint32_t c1) {
    float v0 = c0 ? side_value(s0, c0) : 0.0f;
    float v1 = c1 ? side_value(s1, c1) : 0.0f;
    if (!c0) v0 = c1 ? v1 : 0.0f;
    if (!c1) v1 = c0 ? v0 : 0.0f;
    return make_float2(v0, v1);
}

// leaves: value straight from their own sums (used when the tree is a single leaf)
__global__ void k_leaf_values(uint32_t off, uint32_t n, const ulonglong2* __restrict__ acc_sum,
                              const uint2* __restrict__ acc_cnt, float2* __restrict__ value) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const ulonglong2 s = acc_sum[off + j];
    const uint2 c = acc_cnt[off + j];
    value[off + j] = node_values(s.x, c.x, s.y, c.y);
}

// one inner level: own records + children's sums routed to the parent side
// their normal agrees with; when the children are leaves their values are
// written here too (a leaf's value comes from its own sums)
__global__ void k_reduce_level(uint32_t off, uint32_t n, int children_are_leaves, const Node* __restrict__ node,
                               const uint8_t* __restrict__ route, const ulonglong2* __restrict__ acc_sum,
                               const uint2* __restrict__ acc_cnt, ulonglong2* __restrict__ tot_sum,
                               uint2* __restrict__ tot_cnt, float2* __restrict__ value) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t id = off + j;
    const Node nd = node[id];
    const ulonglong2 own = acc_sum[id];
    const uint2 ownc = acc_cnt[id];
    unsigned long long s0 = own.x, s1 = own.y;
    uint32_t c0 = ownc.x, c1 = ownc.y;
    const ulonglong2* csum = children_are_leaves ? acc_sum : tot_sum;
    const uint2* ccnt = children_are_leaves ? acc_cnt : tot_cnt;
    const int m = __popc(nd.mask);
    for (int k = 0; k < m; ++k) {
        const uint32_t ch = nd.first_child + k;
        const uint32_t r = route[ch];
        const ulonglong2 cs = csum[ch];
        const uint2 cc = ccnt[ch];
        if (children_are_leaves) value[ch] = node_values(cs.x, cc.x, cs.y, cc.y);
        if (!(r & 1u)) { s0 += cs.x; c0 += cc.x; } else { s1 += cs.x; c1 += cc.x; }
        if (!(r & 2u)) { s0 += cs.y; c0 += cc.y; } else { s1 += cs.y; c1 += cc.y; }
    }
    tot_sum[id] = make_ulonglong2(s0, s1);
    tot_cnt[id] = make_uint2(c0, c1);
    value[id] = node_values(s0, c0, s1, c1);
}

// n_dev: optional device count of valid records (the first min(*n_dev, n))
int accumulate(wfpg_svo* s, const float* pos, const float* wout, const float* L, uint32_t n, cudaStream_t st,
               const uint32_t* n_dev) {
    const int T = 256;
    if (n > 0) {
        AccArgs A;
        A.node = s->node;
        A.normal = s->normal;
        A.D = s->D;
        for (int a = 0; a < 3; ++a) A.lo[a] = s->lo[a];
        A.scale = s->scale;
        WFPG_LAUNCH(k_accumulate, div_up(n, T), T, 0, st, A, pos, wout, L, n, n_dev, s->acc_sum, s->acc_cnt);
    }
    const int D = s->D;
    const auto* as = reinterpret_cast<const ulonglong2*>(s->acc_sum);
    const auto* ac = reinterpret_cast<const uint2*>(s->acc_cnt);
    auto* ts = reinterpret_cast<ulonglong2*>(s->tot_sum);
    auto* tc = reinterpret_cast<uint2*>(s->tot_cnt);
    if (D == 0) {
        const uint32_t nl = s->level_off[D + 1] - s->level_off[D];
        WFPG_LAUNCH(k_leaf_values, div_up(nl, T), T, 0, st, s->level_off[D], nl, as, ac, s->value);
    }
    for (int l = D - 1; l >= 0; --l) {
        const uint32_t cnt = s->level_off[l + 1] - s->level_off[l];
        WFPG_LAUNCH(k_reduce_level, div_up(cnt, T), T, 0, st, s->level_off[l], cnt, l + 1 == D, s->node, s->route,
                    as, ac, ts, tc, s->value);
    }
    return launch_status();
}

}  // namespace wfpg
