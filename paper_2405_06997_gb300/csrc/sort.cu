// Device-wide exclusive scan and stable LSD radix sort (8-bit digits).
//
// Radix pass = (1) per-tile digit histograms, (2) one exclusive scan over the
// digit-major histogram table, which yields every (digit, tile) output base,
// (3) a stable scatter: each tile ranks its keys round by round (256 keys per
// round, lane order inside a warp from __match_any_sync, warp order from a
// per-round prefix over per-warp digit counts).
#include "common.cuh"
#include "sort.cuh"

namespace wfpg {

// ---------------------------------------------------------------------------
// block-wide exclusive scan of one value per thread (256 threads)
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* warp_tot, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, k);
        if (lane >= k) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < (kScanBlock / 32) ? warp_tot[lane] : 0u;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, k);
            if (lane >= k) t += y;
        }
        if (lane < (kScanBlock / 32)) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? warp_tot[w - 1] : 0u) + (x - v);
    *total = warp_tot[kScanBlock / 32 - 1];
    return before;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const uint32_t* __restrict__ in,
                                                            uint32_t n, uint32_t* __restrict__ sums) {
    __shared__ uint32_t wt[kScanBlock / 32];
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t tot;
    block_exclusive(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_down(const uint32_t* in, uint32_t* out, uint32_t n,
                                                          const uint32_t* __restrict__ block_base,
                                                          uint32_t* total_dev) {
    __shared__ uint32_t wt[kScanBlock / 32];
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t tot;
    uint32_t run = block_exclusive(s, wt, &tot) + (block_base ? block_base[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (total_dev && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanBlock - 1) *total_dev = run;
}

size_t scan_workspace_bytes(uint32_t n) {
    size_t b = 0;
    uint32_t m = n;
    while (m > (uint32_t)kScanTile) {
        m = div_up(m, kScanTile);
        b += arena_bytes<uint32_t>(m);
    }
    return b + 256;
}

void scan_exclusive(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total_dev, Arena& ws,
                    cudaStream_t s) {
    if (n == 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, 4, s);
        return;
    }
    const uint32_t blocks = div_up(n, kScanTile);
    if (blocks == 1) {
        WFPG_LAUNCH(k_scan_down, 1, kScanBlock, 0, s, in, out, n, nullptr, total_dev);
        return;
    }
    uint32_t* sums = ws.take<uint32_t>(blocks);
    WFPG_LAUNCH(k_scan_reduce, blocks, kScanBlock, 0, s, in, n, sums);
    scan_exclusive(sums, sums, blocks, nullptr, ws, s);
    WFPG_LAUNCH(k_scan_down, blocks, kScanBlock, 0, s, in, out, n, sums, total_dev);
}

// ---------------------------------------------------------------------------
// per-tile digit counts: each warp counts into its own sub-histogram (keys that
// are already partly sorted by earlier passes would otherwise pile onto a few
// shared-memory counters), then the sub-histograms are summed per digit
template <typename K>
__global__ void __launch_bounds__(kSortBlock) k_radix_hist(const K* __restrict__ keys, uint32_t n,
                                                           int shift, uint32_t* __restrict__ hist,
                                                           uint32_t tiles) {
    constexpr int W = kSortBlock / 32;
    __shared__ uint32_t h[W][256];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < W * 256; i += kSortBlock) (&h[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t e = base + r * kSortBlock + threadIdx.x;
        if (e < n) atomicAdd(&h[w][(uint32_t)(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t sum = 0u;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) sum += h[ww][threadIdx.x];
    hist[threadIdx.x * tiles + blockIdx.x] = sum;
}

template <typename K, bool kVals>
__global__ void __launch_bounds__(kSortBlock) k_radix_scatter(const K* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin,
                                                              K* __restrict__ kout,
                                                              uint32_t* __restrict__ vout, uint32_t n,
                                                              int shift, const uint32_t* __restrict__ offs,
                                                              uint32_t tiles) {
    constexpr int W = kSortBlock / 32;
    __shared__ uint32_t whist[W][257];
    __shared__ uint32_t wbase[W][257];
    __shared__ uint32_t run[256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < W * 257; i += kSortBlock) (&whist[0][0])[i] = 0u;
    run[tid] = offs[tid * tiles + blockIdx.x];
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t e = base + r * kSortBlock + tid;
        const bool valid = e < n;
        const K k = valid ? kin[e] : (K)0;
        const uint32_t v = (kVals && valid) ? vin[e] : 0u;
        const int d = valid ? (int)((uint32_t)(k >> shift) & 255u) : 256;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (rank == 0) whist[w][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = run[tid];
#pragma unroll
            for (int ww = 0; ww < W; ++ww) {
                const uint32_t t = whist[ww][tid];
                wbase[ww][tid] = acc;
                acc += t;
                whist[ww][tid] = 0u;
            }
            run[tid] = acc;
            if (tid < W) whist[tid][256] = 0u;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wbase[w][d] + rank;
            kout[pos] = k;
            if (kVals) vout[pos] = v;
        }
    }
}

size_t radix_sort_workspace_bytes(uint32_t n) {
    const uint32_t tiles = div_up(n ? n : 1, kSortTile);
    return arena_bytes<uint32_t>((size_t)tiles * 256) + scan_workspace_bytes(tiles * 256);
}

template <typename K, bool kVals>
static void radix_sort_impl(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, uint32_t n,
                            int bits, Arena& ws, cudaStream_t s, K** kres, uint32_t** vres) {
    *kres = keys;
    if (vres) *vres = vals;
    if (n <= 1 || bits <= 0) return;
    const uint32_t tiles = div_up(n, kSortTile);
    const size_t mark = ws.used;
    uint32_t* hist = ws.take<uint32_t>((size_t)tiles * 256);
    K* a = keys;
    K* b = keys_alt;
    uint32_t* va = vals;
    uint32_t* vb = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        WFPG_LAUNCH(k_radix_hist<K>, tiles, kSortBlock, 0, s, a, n, shift, hist, tiles);
        const size_t m2 = ws.used;
        scan_exclusive(hist, hist, tiles * 256, nullptr, ws, s);
        ws.used = m2;
        auto scatter = k_radix_scatter<K, kVals>;
        WFPG_LAUNCH(scatter, tiles, kSortBlock, 0, s, a, va, b, vb, n, shift, hist, tiles);
        K* t = a;
        a = b;
        b = t;
        uint32_t* tv = va;
        va = vb;
        vb = tv;
    }
    ws.used = mark;
    *kres = a;
    if (vres) *vres = va;
}

void radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t n, int bits, Arena& ws,
                    cudaStream_t s, uint64_t** sorted) {
    radix_sort_impl<uint64_t, false>(keys, keys_alt, nullptr, nullptr, n, bits, ws, s, sorted, nullptr);
}

void radix_sort_pairs_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                          uint32_t n, int bits, Arena& ws, cudaStream_t s, uint32_t** keys_out,
                          uint32_t** vals_out) {
    radix_sort_impl<uint32_t, true>(keys, keys_alt, vals, vals_alt, n, bits, ws, s, keys_out, vals_out);
}

}  // namespace wfpg
