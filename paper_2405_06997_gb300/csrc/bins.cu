// Positional binning, Partition-S (Alg. 2, Sec. 3.4), its run-length
// stand-in, and SelectOrigin (Sec. 3 "Implementation").
#include "common.cuh"
#include "sort.cuh"
#include "svo.cuh"

namespace wfpg {

struct LevelOffsets {
    uint32_t off[WFPG_MAX_DEPTH + 2];
};

__device__ __forceinline__ int level_of(const LevelOffsets& L, int D, uint32_t node) {
    int l = 0;
    while (l < D && node >= L.off[l + 1]) ++l;
    return l;
}

// number of valid rays: the device count when given (at most the capacity n)
__device__ __forceinline__ uint32_t ray_count(uint32_t n, const uint32_t* n_dev) {
    return n_dev ? min(*n_dev, n) : n;
}

// DescendLeaf + AtomicAdd: each ray counts at the deepest node holding it
__global__ void __launch_bounds__(256) k_bin_descend(const Node* __restrict__ nodes, int D, float lox, float loy,
                                                     float loz, float scale, const float* __restrict__ pos, uint32_t n,
                                                     const uint32_t* __restrict__ n_dev, uint32_t* __restrict__ ray_node,
                                                     uint32_t* __restrict__ count) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < ray_count(n, n_dev);
    uint32_t nd = 0xffffffffu;
    if (valid) {
        int c[3];
        c[0] = grid_index(pos[3 * (size_t)i + 0], lox, scale, D);
        c[1] = grid_index(pos[3 * (size_t)i + 1], loy, scale, D);
        c[2] = grid_index(pos[3 * (size_t)i + 2], loz, scale, D);
        int lvl;
        nd = descend(nodes, c, D, &lvl);
        ray_node[i] = nd;
    }
    // neighbouring rays mostly share a node: one atomic per distinct node of the warp
    const uint32_t peers = __match_any_sync(0xffffffffu, nd);
    const uint32_t lane = threadIdx.x & 31u;
    if (valid && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&count[nd], (uint32_t)__popc(peers));
}

// one level of the bottom-up ray totals; bit 31 marks the node
__global__ void k_bin_level(uint32_t off, uint32_t n, int is_leaf_level, int is_lmin, uint32_t c_ray,
                            const Node* __restrict__ nodes, const uint32_t* __restrict__ count,
                            uint32_t* __restrict__ total) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t id = off + j;
    uint32_t T = count[id];
    if (!is_leaf_level) {
        const Node nd = nodes[id];
        const int m = __popc(nd.mask);
        for (int k = 0; k < m; ++k) T += total[nd.first_child + k] & 0x7fffffffu;
    }
    const bool mark = (T >= c_ray) || is_lmin;
    total[id] = T | (mark ? 0x80000000u : 0u);
}

// AscendAndFindMarked
__global__ void __launch_bounds__(256) k_bin_ascend(uint32_t* __restrict__ ray_node, uint32_t n,
                                                    const uint32_t* __restrict__ n_dev, LevelOffsets L, int D,
                                                    int l_min, const uint32_t* __restrict__ parent,
                                                    const uint32_t* __restrict__ total, uint32_t* __restrict__ used) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ray_count(n, n_dev)) return;
    uint32_t nd = ray_node[i];
    if (level_of(L, D, nd) >= l_min) {
        while (!(total[nd] >> 31)) nd = parent[nd];
    }
    ray_node[i] = nd;
    used[nd] = 1u;
}

// rays past the device count get the largest key, so a stable sort leaves
// them after every valid ray
__global__ void __launch_bounds__(256) k_bin_ids(const uint32_t* __restrict__ bin_node, uint32_t n,
                                                 const uint32_t* __restrict__ n_dev,
                                                 const uint32_t* __restrict__ rank, uint32_t* __restrict__ bin_of_ray,
                                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vals[i] = i;
    if (i >= ray_count(n, n_dev)) {
        keys[i] = 0xffffffffu;
        return;
    }
    const uint32_t b = rank[bin_node[i]];
    bin_of_ray[i] = b;
    keys[i] = b;
}

// bin_offset[b] = first sorted position of bin b; bin_offset[n_bins] = n
__global__ void __launch_bounds__(256) k_bin_offsets(const uint32_t* __restrict__ sorted_bins, uint32_t n_cap,
                                                     const uint32_t* __restrict__ n_dev,
                                                     uint32_t* __restrict__ bin_offset, uint32_t bin_cap,
                                                     const uint32_t* __restrict__ n_bins_dev,
                                                     uint32_t* __restrict__ status) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = ray_count(n_cap, n_dev);
    if (p == 0) {
        const uint32_t nb = *n_bins_dev;
        if (nb <= bin_cap) bin_offset[nb] = n;
        else atomicOr(status, (uint32_t)WFPG_STATUS_BIN_CAPACITY);
    }
    if (p >= n) return;
    const uint32_t k = sorted_bins[p];
    if ((p == 0 || sorted_bins[p - 1] != k) && k <= bin_cap) bin_offset[k] = p;
}

// SelectOrigin: bin b takes position floor(u24 * size / 2^24) of its run
__global__ void k_bin_origins(const uint32_t* __restrict__ bin_offset, const uint32_t* __restrict__ ray_order,
                              uint32_t n_cap, const uint32_t* __restrict__ n_dev,
                              const uint32_t* __restrict__ n_bins_dev, uint32_t bin_cap, uint64_t seed,
                              uint32_t frame_arg, const uint32_t* __restrict__ frame_dev,
                              uint32_t* __restrict__ origin_ray) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = ray_count(n_cap, n_dev);
    const uint32_t frame = frame_dev ? *frame_dev : frame_arg;
    const uint32_t nb = min(*n_bins_dev, bin_cap);
    if (b >= nb) return;
    const uint32_t lo = bin_offset[b], hi = bin_offset[b + 1];
    if (hi <= lo || lo >= n) {
        origin_ray[b] = kNone;
        return;
    }
    const uint64_t u = uniform24(purpose(seed, kOriginPurpose), bin_stream(frame, b), 0);
    const uint64_t k = (u * (uint64_t)(hi - lo)) >> 24;
    const uint64_t p = lo + k;
    origin_ray[b] = p < n ? ray_order[p] : kNone;
}

// ---------------------------------------------------------------- runs mode
__global__ void __launch_bounds__(256) k_runs_keys(const float* __restrict__ pos, const float* __restrict__ nrm,
                                                   uint32_t n, const uint32_t* __restrict__ n_dev, float lox, float loy,
                                                   float loz, float scale, int D, uint32_t* __restrict__ keys,
                                                   uint32_t* __restrict__ vals) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vals[i] = i;
    if (i >= ray_count(n, n_dev)) {
        keys[i] = 0xffffffffu;
        return;
    }
    const int q = D < 6 ? D : 6;
    const uint32_t cx = (uint32_t)grid_index(pos[3 * (size_t)i + 0], lox, scale, D) >> (D - q);
    const uint32_t cy = (uint32_t)grid_index(pos[3 * (size_t)i + 1], loy, scale, D) >> (D - q);
    const uint32_t cz = (uint32_t)grid_index(pos[3 * (size_t)i + 2], loz, scale, D) >> (D - q);
    const uint32_t oct = (nrm[3 * (size_t)i + 0] < 0.0f ? 1u : 0u) | (nrm[3 * (size_t)i + 1] < 0.0f ? 2u : 0u) |
                         (nrm[3 * (size_t)i + 2] < 0.0f ? 4u : 0u);
    keys[i] = (uint32_t)(morton3(cx, cy, cz) << 3) | oct;
}

__global__ void k_runs_check(const uint32_t* __restrict__ sizes, uint32_t nb, const uint32_t* __restrict__ total,
                             uint32_t n_cap, const uint32_t* __restrict__ n_dev, uint32_t* __restrict__ bin_offset,
                             uint32_t* __restrict__ n_bins_dev, uint32_t* __restrict__ status) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = ray_count(n_cap, n_dev);
    if (b == 0) {
        bin_offset[nb] = *total;
        *n_bins_dev = nb;
        if (*total != n) atomicOr(status, (uint32_t)WFPG_STATUS_RUN_SIZES);
    }
    if (b < nb && sizes[b] == 0) atomicOr(status, (uint32_t)WFPG_STATUS_RUN_SIZES);
}

__global__ void __launch_bounds__(256) k_runs_bins(const uint32_t* __restrict__ bin_offset, uint32_t nb,
                                                   const uint32_t* __restrict__ ray_order, uint32_t n_cap,
                                                   const uint32_t* __restrict__ n_dev,
                                                   uint32_t* __restrict__ bin_of_ray) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = ray_count(n_cap, n_dev);
    if (p >= n) return;
    uint32_t lo = 0, hi = nb;  // last b with bin_offset[b] <= p
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (bin_offset[mid] <= p) lo = mid;
        else hi = mid;
    }
    const uint32_t r = ray_order[p];
    if (r < n) bin_of_ray[r] = lo;
}

// ---------------------------------------------------------------------------
static int bits_for(uint64_t max_value) {
    int b = 0;
    while (b < 32 && (max_value >> b) != 0) ++b;
    return b;
}

// The sort alternates between its two value buffers, one 8-bit pass each, so
// the ray order ends in the caller's ray_order without a copy when the pass
// count picks which buffer the ray indices start in.
static uint32_t* sort_values_start(int bits, uint32_t* ray_order, uint32_t* vals) {
    const int b = bits < 32 ? bits : 32;
    return ((b + 7) / 8) % 2 == 0 ? ray_order : vals;
}

size_t bin_workspace_bytes(const wfpg_svo* s, uint32_t n, int mode, uint32_t n_sizes) {
    size_t b = 0;
    b += 3 * arena_bytes<uint32_t>(n);                     // keys, keys_alt, vals (ray_order is the 4th)
    b += radix_sort_workspace_bytes(n);
    if (mode == WFPG_BIN_PARTITION_S) {
        b += arena_bytes<uint32_t>(n);                     // ray_node
        b += 3 * arena_bytes<uint32_t>(s->n_nodes);        // count, total, used/rank
        b += scan_workspace_bytes(s->n_nodes);
    } else {
        b += scan_workspace_bytes((n > n_sizes ? n : n_sizes) + 1) + arena_bytes<uint32_t>(1);
    }
    return b + 1024;
}

int bin_rays_impl(const wfpg_svo* s, const float* pos, const float* nrm, uint32_t n, const wfpg_bin_params* p,
                  const uint32_t* sizes, uint32_t* bin_of_ray, uint32_t* ray_order, uint32_t* bin_offset,
                  uint32_t* origin_ray, uint32_t bin_cap, uint32_t* n_bins_dev, void* workspace, size_t ws_bytes,
                  cudaStream_t st, const uint32_t* frame_dev) {
    const uint32_t* nd = p->n_dev;  // optional device count of valid rays (<= n)
    const int T = 256;
    const int D = s->D;
    Arena ws{static_cast<char*>(workspace), ws_bytes, 0, false};
    uint32_t* keys = ws.take<uint32_t>(n);
    uint32_t* keys_alt = ws.take<uint32_t>(n);
    uint32_t* vals = ws.take<uint32_t>(n);
    if (ws.overflow) return WFPG_ERR_INVALID_ARG;
    uint32_t* skeys = nullptr;
    uint32_t* svals = nullptr;
    if (p->mode == WFPG_BIN_PARTITION_S) {
        const int l_min = p->l_min < 0 ? 0 : (p->l_min > D ? D : p->l_min);
        uint32_t* ray_node = ws.take<uint32_t>(n);
        uint32_t* count = ws.take<uint32_t>(s->n_nodes);
        uint32_t* total = ws.take<uint32_t>(s->n_nodes);
        uint32_t* used = ws.take<uint32_t>(s->n_nodes);
        if (ws.overflow) return WFPG_ERR_INVALID_ARG;
        cudaMemsetAsync(count, 0, 4 * (size_t)s->n_nodes, st);
        cudaMemsetAsync(used, 0, 4 * (size_t)s->n_nodes, st);
        if (n > 0)
            WFPG_LAUNCH(k_bin_descend, div_up(n, T), T, 0, st, s->node, D, s->lo[0], s->lo[1], s->lo[2], s->scale, pos, n,
                        nd, ray_node, count);
        for (int l = D; l >= l_min; --l) {
            const uint32_t cnt = s->level_off[l + 1] - s->level_off[l];
            WFPG_LAUNCH(k_bin_level, div_up(cnt, T), T, 0, st, s->level_off[l], cnt, l == D, l == l_min, p->c_ray, s->node,
                                                      count, total);
        }
        LevelOffsets L;
        for (int l = 0; l < WFPG_MAX_DEPTH + 2; ++l) L.off[l] = s->level_off[l];
        if (n > 0)
            WFPG_LAUNCH(k_bin_ascend, div_up(n, T), T, 0, st, ray_node, n, nd, L, D, l_min, s->parent, total, used);
        scan_exclusive(used, used, s->n_nodes, n_bins_dev, ws, st);
        const uint64_t max_bins = n < s->n_nodes ? n : s->n_nodes;
        const int bits = bits_for(max_bins);
        uint32_t* v0 = sort_values_start(bits, ray_order, vals);
        uint32_t* v1 = v0 == ray_order ? vals : ray_order;
        if (n > 0)
            WFPG_LAUNCH(k_bin_ids, div_up(n, T), T, 0, st, ray_node, n, nd, used, bin_of_ray, keys, v0);
        radix_sort_pairs_u32(keys, keys_alt, v0, v1, n, bits, ws, st, &skeys, &svals, s->status);
        if (ws.overflow) return WFPG_ERR_INVALID_ARG;  // the sort's look-back words did not fit
        if (n > 0 && svals != ray_order)
            cudaMemcpyAsync(ray_order, svals, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st);
        WFPG_LAUNCH(k_bin_offsets, div_up(n + 1, T), T, 0, st, skeys, n, nd, bin_offset, bin_cap, n_bins_dev, s->status);
    } else {
        if (p->n_sizes > bin_cap) return WFPG_ERR_CAPACITY;
        const int q = D < 6 ? D : 6;
        uint32_t* tot = ws.take<uint32_t>(1);
        if (ws.overflow) return WFPG_ERR_INVALID_ARG;
        const int bits = 3 * q + 3;
        uint32_t* v0 = sort_values_start(bits, ray_order, vals);
        uint32_t* v1 = v0 == ray_order ? vals : ray_order;
        if (n > 0)
            WFPG_LAUNCH(k_runs_keys, div_up(n, T), T, 0, st, pos, nrm, n, nd, s->lo[0], s->lo[1], s->lo[2], s->scale, D,
                        keys, v0);
        radix_sort_pairs_u32(keys, keys_alt, v0, v1, n, bits, ws, st, &skeys, &svals, s->status);
        if (ws.overflow) return WFPG_ERR_INVALID_ARG;  // the sort's look-back words did not fit
        if (n > 0 && svals != ray_order)
            cudaMemcpyAsync(ray_order, svals, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st);
        scan_exclusive(sizes, bin_offset, p->n_sizes, tot, ws, st);
        WFPG_LAUNCH(k_runs_check, div_up(p->n_sizes + 1, T), T, 0, st, sizes, p->n_sizes, tot, n, nd, bin_offset,
                    n_bins_dev, s->status);
        if (n > 0 && p->n_sizes > 0)
            WFPG_LAUNCH(k_runs_bins, div_up(n, T), T, 0, st, bin_offset, p->n_sizes, ray_order, n, nd, bin_of_ray);
    }
    if (bin_cap > 0)
        WFPG_LAUNCH(k_bin_origins, div_up(bin_cap, T), T, 0, st, bin_offset, ray_order, n, nd, n_bins_dev, bin_cap,
                    p->seed, p->frame, frame_dev, origin_ray);
    return launch_status();
}

}  // namespace wfpg
