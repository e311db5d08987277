// Device-wide exclusive scan and stable LSD radix sorts (8-bit digits).
//
// 64-bit keys (the SVO builder): radix pass = (1) per-tile digit histograms,
// (2) one exclusive scan over the digit-major histogram table, which yields
// every (digit, tile) output base, (3) a stable scatter: each tile ranks its
// keys round by round (256 keys per round, lane order inside a warp from
// __match_any_sync, warp order from a per-round prefix over per-warp digit
// counts).  32-bit keys with values (the binning): one launch per pass, each
// warp ranking its own run of the tile's keys, the tile bases found by
// decoupled look-back (below).
#include <algorithm>
#include <utility>

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

// ---------------------------------------------------------------------------
// One-sweep LSD radix sort of 32-bit keys with values (8-bit digits).  One
// kernel counts the digits of every pass over the whole input; then one kernel
// per pass ranks each tile's keys (stable: each warp ranks 512 consecutive
// keys against its own digit counters, with warp barriers only, then one block
// barrier turns the warps' counts into their bases), publishes the tile's
// digit counts, adds up the counts of all earlier tiles by looking back over
// what they published (decoupled look-back), and scatters.  A block takes its
// tile from a ticket counter, so it only ever waits on tiles held by blocks
// that started before it; every wait is bounded.
//
// Look-back word of (tile, digit): bits 0..26 a count, bits 27..29 the pass + 1
// (0: nothing published in this sort yet), bit 30 the tile's own count, bit 31
// the count of this tile and all tiles before it.
constexpr uint32_t kLbCount = (1u << 27) - 1u;
constexpr int kLbTagShift = 27;
constexpr uint32_t kLbTagMask = 7u << kLbTagShift;
constexpr uint32_t kLbAggregate = 1u << 30, kLbInclusive = 1u << 31;
constexpr int kSweepMaxPasses = 4;
constexpr uint32_t kLbSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// digit counts of passes 0 .. passes - 1 over all n keys (per-warp sub-histograms)
__global__ void __launch_bounds__(kSortBlock) k_sweep_hist(const uint32_t* __restrict__ keys, uint32_t n,
                                                           int passes, uint32_t* __restrict__ ghist) {
    constexpr int W = kSortBlock / 32;
    __shared__ uint32_t h[W][kSweepMaxPasses][256];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < W * kSweepMaxPasses * 256; i += kSortBlock) (&h[0][0][0])[i] = 0u;
    __syncthreads();
    for (uint32_t e = blockIdx.x * kSortBlock + threadIdx.x; e < n; e += gridDim.x * kSortBlock) {
        const uint32_t k = keys[e];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[w][p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        uint32_t sum = 0u;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) sum += h[ww][p][threadIdx.x];
        if (sum) atomicAdd(&ghist[p * 256 + threadIdx.x], sum);
    }
}

template <bool kVals>
__global__ void __launch_bounds__(kSortBlock) k_sweep_pass(const uint32_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ kout,
                                                           uint32_t* __restrict__ vout, uint32_t n, int pass,
                                                           const uint32_t* __restrict__ ghist, uint32_t* look,
                                                           uint32_t* ticket, uint32_t* status) {
    constexpr int W = kSortBlock / 32;
    constexpr int kWarpKeys = 32 * kSortItems;  // each warp ranks 512 consecutive keys of the tile
    __shared__ uint32_t whist[W][256];          // per warp: its keys of each digit so far, then its base
    __shared__ uint32_t start[256];
    __shared__ uint32_t wt[kScanBlock / 32];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int shift = 8 * pass;
    const uint32_t tag = (uint32_t)(pass + 1) << kLbTagShift;
    if (tid == 0) s_tile = atomicAdd(ticket + pass, 1u);
    for (int i = tid; i < W * 256; i += kSortBlock) (&whist[0][0])[i] = 0u;
    // where each digit's keys start in the output (exclusive scan of the pass's counts)
    uint32_t total;
    const uint32_t g0 = block_exclusive(ghist[pass * 256 + tid], wt, &total);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t base = tile * kSortTile + (uint32_t)w * kWarpKeys;
    uint32_t* wh = whist[w];
    // ranks inside the warp's keys (key order: round by round, lanes in order); only this warp
    // touches its row, so warp barriers suffice
    uint32_t kr[kSortItems], vr[kSortItems], loc[kSortItems];  // loc: digit << 16 | offset among the warp's keys of it
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t e = base + r * 32 + lane;
        const bool valid = e < n;
        const uint32_t k = valid ? kin[e] : 0u;
        kr[r] = k;
        vr[r] = (kVals && valid) ? vin[e] : 0u;
        const int d = valid ? (int)((k >> shift) & 255u) : 256;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0u;
        if (valid && lane == leader) {
            before = wh[d];
            wh[d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        __syncwarp();
        loc[r] = valid ? (((uint32_t)d << 16) | (before + __popc(peers & lt))) : 0xFFFFFFFFu;
    }
    __syncthreads();
    // thread t: digit t.  Each warp's base among the tile's keys of it, and the tile's count.
    uint32_t run = 0u;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
        const uint32_t t = whist[ww][tid];
        whist[ww][tid] = run;
        run += t;
    }
    // thread t: digit t.  Publish this tile's count, add up the earlier tiles' counts, publish the sum.
    const uint32_t cnt = run;
    uint32_t* mine = look + (size_t)tile * 256 + tid;
    uint32_t excl = 0u;
    bool ok = true;
    if (tile == 0) {
        st_release_u32(mine, tag | kLbInclusive | cnt);
    } else {
        st_release_u32(mine, tag | kLbAggregate | cnt);
        int p = (int)tile - 1;
        uint32_t spins = 0u;
        while (p >= 0) {
            const uint32_t v = ld_acquire_u32(look + (size_t)p * 256 + tid);
            if ((v & kLbTagMask) != tag) {  // that tile has not published yet
                if (++spins > kLbSpinLimit) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl += v & kLbCount;
            if (v & kLbInclusive) break;
            --p;
        }
        st_release_u32(mine, tag | kLbInclusive | ((excl + cnt) & kLbCount));
    }
    if (!ok && status) atomicOr(status, (uint32_t)WFPG_STATUS_WAIT_TIMEOUT);
    start[tid] = g0 + excl;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (loc[r] != 0xFFFFFFFFu) {
            const uint32_t dg = loc[r] >> 16;
            const uint32_t pos = start[dg] + whist[w][dg] + (loc[r] & 0xFFFFu);
            if (pos < n) {  // always, unless a wait ran out above
                kout[pos] = kr[r];
                if (kVals) vout[pos] = vr[r];
            }
        }
    }
}

size_t radix_sort_workspace_bytes(uint32_t n) {
    const uint32_t tiles = div_up(n ? n : 1, kSortTile);
    const size_t lsd = arena_bytes<uint32_t>((size_t)tiles * 256) + scan_workspace_bytes(tiles * 256);
    const size_t sweep = arena_bytes<uint32_t>((size_t)kSweepMaxPasses * 256 + kSweepMaxPasses + (size_t)tiles * 256);
    return lsd > sweep ? lsd : sweep;
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
                          uint32_t** vals_out, uint32_t* status) {
    *keys_out = keys;
    *vals_out = vals;
    if (n <= 1 || bits <= 0) return;
    if (n > kLbCount) {  // counts would not fit the look-back words: per-pass histograms and scans
        radix_sort_impl<uint32_t, true>(keys, keys_alt, vals, vals_alt, n, bits, ws, s, keys_out, vals_out);
        return;
    }
    const int passes = (bits < 32 ? bits : 32) / 8 + ((bits < 32 ? bits : 32) % 8 ? 1 : 0);
    const uint32_t tiles = div_up(n, kSortTile);
    const size_t mark = ws.used;
    uint32_t* ghist = ws.take<uint32_t>((size_t)kSweepMaxPasses * 256 + kSweepMaxPasses + (size_t)tiles * 256);
    if (!ghist) {
        ws.used = mark;
        return;
    }
    uint32_t* ticket = ghist + kSweepMaxPasses * 256;
    uint32_t* look = ticket + kSweepMaxPasses;
    cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * ((size_t)kSweepMaxPasses * 256 + kSweepMaxPasses + (size_t)tiles * 256), s);
    const uint32_t hgrid = std::min<uint32_t>(div_up(n, kSortBlock * 16), 1024u);
    WFPG_LAUNCH(k_sweep_hist, hgrid, kSortBlock, 0, s, keys, n, passes, ghist);
    uint32_t* a = keys;
    uint32_t* b = keys_alt;
    uint32_t* va = vals;
    uint32_t* vb = vals_alt;
    for (int pass = 0; pass < passes; ++pass) {
        WFPG_LAUNCH(k_sweep_pass<true>, tiles, kSortBlock, 0, s, a, va, b, vb, n, pass, ghist, look, ticket, status);
        std::swap(a, b);
        std::swap(va, vb);
    }
    ws.used = mark;
    *keys_out = a;
    *vals_out = va;
}

}  // namespace wfpg
