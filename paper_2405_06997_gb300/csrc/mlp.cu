// The learned proposal (a project addition; the paper has no counterpart):
// an MLP 78 -> 64 -> 64 -> 64 -> 1024 (ReLU) whose softmax over the 32 x 32
// octahedral cells proposes a bin's directional distribution, trained online
// against the SVO-traced fields of Alg. 3 with KL(q || softmax(z)).
//
// Every layer, forward and backward, is one tcgen05 GEMM on bfloat16 operands
// with float32 accumulation in tensor memory:
//   forward   H1 = relu(X W1^T + b1), H2, H3 likewise, Z = H3 W4^T + b4
//   backward  G4 = (softmax(Z) - q) / n; dW4 = G4^T H3, dA3 = (G4 W4) o [H3 > 0],
//             dW3 = dA3^T H2, dA2 = (dA3 W3) o [H2 > 0], ... , dW1 = dA1^T X
// All GEMMs are "TN": D[M x N] = A[M x K] B[N x K]^T with both operands
// K-contiguous, so the backward uses transposed copies (written by the
// forward epilogues and the weight-conversion kernel).  Weight gradients
// reduce over the batch with split-K: per-split partial tiles, then one summing pass.  Adam updates
// float32 master weights, then bfloat16 copies are refreshed.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>

#include "common.cuh"
#include "svo.cuh"
#include "tc.cuh"

typedef __nv_bfloat16 bf16;

namespace wfpg {
int field_pdf_impl(const float* field, int N, const uint32_t* n_bins_dev, uint32_t bin_cap, float* pdf,
                   float* cdf_row, float* cdf_marg, cudaStream_t st, int blur = 0);
int set_last_error(int code, const std::string& msg);
}  // namespace wfpg

using namespace wfpg;

namespace {

constexpr int kIn = 80, kHid = 64, kOut = 1024;
constexpr int kFeatIn = 78;  // input features (the rest of the 80 columns is padding)
constexpr int kTRows = 80;   // rows of the transposed activations: 64 (or 78 + 2) values, a row of ones, zeros
constexpr size_t kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
                 kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid,
                 kOffB4 = kOffW4 + (size_t)kOut * kHid, kParams = kOffB4 + kOut;

enum Epi { kEpiF32 = 0, kEpiBf16Relu = 1, kEpiPartial = 2, kEpiReluGrad = 3 };

struct GemmArgs {
    const bf16* A;   // [M][lda], K contiguous
    const bf16* B;   // [N][ldb], K contiguous
    int lda, ldb;
    int M, N, K;
    int chunks_per_split;  // K chunks (KChunk<BN>) per blockIdx.z
    int stages;            // shared-memory tile stages, 1 .. kMaxStages
    float* C;              // f32 output [M][ldc] (kEpiF32); per split z: C + z * split_stride (kEpiPartial)
    int ldc;
    size_t split_stride;
    bf16* O;               // bf16 output [M][ldo]
    int ldo;
    bf16* OT;              // optional transposed bf16 output [N][ldot]
    int ldot;
    const float* bias;     // [N] (kEpiF32, kEpiBf16Relu)
    const bf16* act;       // forward activation [M][ldact] (kEpiReluGrad)
    int ldact;
    uint32_t* status;
};

constexpr int kGemmThreads = 128;
constexpr int kMaxStages = 4;  // K chunks in flight: stages - 1 loading while the MMAs of one run

// streaming multiprocessors of the current device
int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}
// K elements per pipeline step: 128 for narrow tiles (more bytes in flight per
// CTA on the long-K weight-gradient GEMMs), 64 for the 256-wide logits tile
template <int BN>
struct KChunk {
    static constexpr int value = BN <= 80 ? 128 : 64;
};

template <int BN>
struct TmemCols {
    static constexpr uint32_t value = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
};

// copy rows [r0, r0 + rows) x k [k0, k0 + KC) of a K-contiguous bf16 matrix into
// the no-swizzle K-major core-matrix layout with asynchronous 16-byte copies (the
// caller commits and waits): 16-byte piece c of row r goes to (r / 8) * (KC * 16)
// + c * 128 + (r % 8) * 16; rows or k past the end read zero.  When NT threads
// cover whole 8-row groups per pass, each thread keeps one piece column and steps
// its source pointer and destination by whole passes (no index arithmetic per
// copy); otherwise the copies are numbered and split.
template <int KC, int NT = kGemmThreads>
__device__ __forceinline__ void load_tile_async(uint8_t* smem, const bf16* g, int ld, int r0, int rows,
                                                int nrows_total, int k0, int K) {
    constexpr int kCpr = KC / 8;  // 16-byte pieces per row
    if constexpr (NT % kCpr == 0 && (NT / kCpr) % 8 == 0) {
        constexpr int kRstep = NT / kCpr;  // rows per pass
        const int c = threadIdx.x % kCpr, rr = threadIdx.x / kCpr;
        const bool kvalid = k0 + c * 8 < K;
        const bf16* src = g + (size_t)(r0 + rr) * ld + k0 + c * 8;
        uint8_t* dst = smem + (rr >> 3) * (KC * 16) + c * 128 + (rr & 7) * 16;
        const size_t step = (size_t)kRstep * ld;
#pragma unroll
        for (int r = rr; r < rows; r += kRstep) {
            const bool valid = kvalid && r0 + r < nrows_total;
            tc::cp_async16(dst, valid ? src : g, valid);
            src += step;
            dst += (kRstep / 8) * (KC * 16);
        }
    } else {
        for (int idx = threadIdx.x; idx < rows * kCpr; idx += NT) {
            const int r = idx / kCpr, c = idx % kCpr;
            const int gr = r0 + r, gk = k0 + c * 8;
            const bool valid = gr < nrows_total && gk < K;
            tc::cp_async16(smem + (r >> 3) * (KC * 16) + c * 128 + (r & 7) * 16, valid ? g + (size_t)gr * ld + gk : g,
                           valid);
        }
    }
}

// byte offset of element (r, k) in a K-major no-swizzle core-matrix tile of KC columns
template <int KC>
__device__ __forceinline__ int cm_off(int r, int k) {
    return (r >> 3) * (KC * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tn(const __grid_constant__ CUtensorMap tma_a,
                                                          const __grid_constant__ CUtensorMap tma_b, GemmArgs g) {
    constexpr int kKChunk = KChunk<BN>::value;
    constexpr int kAtoms = kKChunk / 64;                 // 128-byte swizzle atoms along K per tile
    constexpr int kABytes = 128 * kKChunk * 2, kBBytes = BN * kKChunk * 2;
    constexpr int kStageBytes = kABytes + kBBytes;
    extern __shared__ __align__(1024) uint8_t gemm_smem_raw[];
    // the swizzled tiles need 1024-byte alignment (the launch adds 1 KB of slack)
    uint8_t* gemm_smem = gemm_smem_raw + ((1024u - (tc::smem_addr(gemm_smem_raw) & 1023u)) & 1023u);
    // g.stages stages of (A tile 128 x kKChunk, B tile BN x kKChunk), each the TMA's
    // 128-byte swizzled layout: atom a (K columns 64 a .. 64 a + 63) of the A tile at
    // a * 16 KB, of the B tile at kABytes + a * BN * 128.  Chunk j sits in stage j % S.
    // One thread runs the pipeline: it issues the TMA copies of chunks i + 1 .. i + S - 1
    // while the MMAs of chunk i run, each stage guarded by a full barrier (the copies
    // have landed) and an empty barrier (the MMAs reading it are done).
    const int S = g.stages;
    auto sA = [&](int s) { return gemm_smem + s * kStageBytes; };
    auto sB = [&](int s) { return gemm_smem + s * kStageBytes + kABytes; };
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ uint32_t tmem_base;
    constexpr uint32_t kCols = TmemCols<BN>::value;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int total_chunks = (g.K + kKChunk - 1) / kKChunk;
    const int kc0 = blockIdx.z * g.chunks_per_split;
    const int kc1 = min(total_chunks, kc0 + g.chunks_per_split);
    const int nch = kc1 - kc0;
    if (warp == 0) tc::tmem_alloc(&tmem_base, kCols);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, BN);
    // the k-th use of stage j % S (k = j / S) completes phase k of its barriers
    auto par = [&](int j) { return (uint32_t)(j / S) & 1u; };
    // the ReLU-mask activations of this thread's row, loaded while the pipeline runs
    constexpr int kActQ = EPI == kEpiReluGrad ? BN / 8 : 1;
    uint4 act_pre[kActQ];
    const bool act_vec = EPI == kEpiReluGrad && n0 + BN <= g.N && (g.ldact & 7) == 0 &&
                         ((uintptr_t)g.act & 15) == 0 && m0 + warp * 32 + lane < g.M;
    if constexpr (EPI == kEpiReluGrad) {
        if (act_vec) {
            const uint4* ap = reinterpret_cast<const uint4*>(g.act + (size_t)(m0 + warp * 32 + lane) * g.ldact + n0);
#pragma unroll
            for (int q = 0; q < kActQ; ++q) act_pre[q] = ap[q];
        }
    }
    bool ok = true;
    if (tid == 0) {
        auto issue = [&](int j) {  // the TMA copies of chunk j (x = K offsets: multiples of 64 elements)
            const int s = j % S, k0 = (kc0 + j) * kKChunk;
            tc::mbar_expect_tx(&full[s], (uint32_t)kStageBytes);
#pragma unroll
            for (int at = 0; at < kAtoms; ++at) {
                tc::tma_load_2d(sA(s) + at * (128 * 128), &tma_a, k0 + 64 * at, m0, &full[s]);
                tc::tma_load_2d(sB(s) + at * (BN * 128), &tma_b, k0 + 64 * at, n0, &full[s]);
            }
        };
        const int P = S > 1 ? S - 1 : 1;  // chunks in flight ahead of the MMAs
        int issued = 0, landed = 0;
        for (; issued < P && issued < nch; ++issued) issue(issued);
        for (int i = 0; i < nch; ++i) {
            const int s = i % S;
            if (!tc::mbar_wait(&full[s], par(i))) {
                ok = false;
                break;
            }
            landed = i + 1;
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sA(s)), b0 = tc::smem_addr(sB(s));
#pragma unroll
            for (int k = 0; k < kKChunk / 16; ++k) {
                const uint32_t off = (uint32_t)(k & 3) * 32u;  // 16 K elements = 32 bytes inside the atom
                const uint64_t ad = tc::smem_desc_sw128(a0 + (uint32_t)(k >> 2) * (128 * 128) + off);
                const uint64_t bd = tc::smem_desc_sw128(b0 + (uint32_t)(k >> 2) * (BN * 128) + off);
                tc::mma_bf16(tmem, ad, bd, idesc, (i > 0 || k > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[s]);
            if (issued < nch) {  // refill the stage last read by the MMAs of chunk issued - S
                if (issued - S >= 0 && !tc::mbar_wait(&empty[issued % S], par(issued - S))) {
                    ok = false;
                    break;
                }
                issue(issued++);
            }
        }
        // the last chunk's commit tracks every MMA issued before it
        if (ok && nch > 0) ok = tc::mbar_wait(&empty[(nch - 1) % S], par(nch - 1));
        // after a timeout, let the copies already issued land before the CTA exits
        for (int j = landed; j < issued; ++j) tc::mbar_wait(&full[j % S], par(j));
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok && lane == 0) atomicOr(g.status, (uint32_t)WFPG_STATUS_MMA_TIMEOUT);
    tc::fence_after_sync();
    bool staged = false;
    if (EPI == kEpiF32 && BN == 256 && ok && kc1 > kc0 && m0 + 128 <= g.M && n0 + BN <= g.N && (g.ldc & 3) == 0 &&
        ((uintptr_t)g.C & 15) == 0) {
        // The wide f32 tile (the logits) goes out through shared memory, 64 columns at a
        // time: each thread moves its TMEM row into a padded staging row, then the CTA
        // writes whole 256-byte row segments (a thread per row would scatter every store
        // over 32 rows).  The MMAs have finished reading the operand tiles, so their
        // shared memory holds the staging slice.
        constexpr int kSlice = 64, kLd = kSlice + 4;
        float* stage = reinterpret_cast<float*>(gemm_smem);
        for (int s0 = 0; s0 < BN; s0 += kSlice) {
#pragma unroll
            for (int c = 0; c < kSlice; c += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s0 + c), v);
                float* srow = stage + (warp * 32 + lane) * kLd + c;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    if (g.bias) {
                        const float* bb = g.bias + n0 + s0 + c + 4 * q;
                        o.x += bb[0];
                        o.y += bb[1];
                        o.z += bb[2];
                        o.w += bb[3];
                    }
                    *reinterpret_cast<float4*>(srow + 4 * q) = o;
                }
            }
            __syncthreads();
            for (int it = tid; it < 128 * (kSlice / 4); it += kGemmThreads) {
                const int r = it / (kSlice / 4), c4 = it % (kSlice / 4);
                *reinterpret_cast<float4*>(g.C + (size_t)(m0 + r) * g.ldc + n0 + s0 + 4 * c4) =
                    *reinterpret_cast<const float4*>(stage + r * kLd + 4 * c4);
            }
            __syncthreads();
        }
        staged = true;
    }
    if (ok && kc1 > kc0 && !staged) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row >= g.M) continue;
            // full 16-column chunks of the row-major outputs go out as 16-byte stores
            if (n0 + c0 + 16 <= g.N) {
                if ((EPI == kEpiF32 || EPI == kEpiPartial) && (g.ldc & 3) == 0 && ((uintptr_t)g.C & 15) == 0 &&
                    (EPI != kEpiPartial || (g.split_stride & 3) == 0)) {
                    float* crow = g.C + (EPI == kEpiPartial ? (size_t)blockIdx.z * g.split_stride : 0);
                    float4* cp = reinterpret_cast<float4*>(crow + (size_t)row * g.ldc + n0 + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        if (EPI == kEpiF32 && g.bias) {
                            const float* bb = g.bias + n0 + c0 + 4 * q;
                            o.x += bb[0];
                            o.y += bb[1];
                            o.z += bb[2];
                            o.w += bb[3];
                        }
                        cp[q] = o;
                    }
                    continue;
                }
                if ((EPI == kEpiBf16Relu || EPI == kEpiReluGrad) && (g.ldo & 7) == 0 && ((uintptr_t)g.O & 15) == 0 &&
                    (EPI != kEpiReluGrad || ((g.ldact & 7) == 0 && ((uintptr_t)g.act & 15) == 0))) {
                    float ar[16];  // forward activations of the 16 columns (ReLU gradient mask)
                    if constexpr (EPI == kEpiReluGrad) {
                        const uint4* ap = reinterpret_cast<const uint4*>(g.act + (size_t)row * g.ldact + n0 + c0);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const uint4 a4 = act_vec ? act_pre[c0 / 8 + q] : ap[q];
                            const uint32_t aw[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                ar[8 * q + 2 * h] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(aw[h] & 0xffffu)));
                                ar[8 * q + 2 * h + 1] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(aw[h] >> 16)));
                            }
                        }
                    }
                    uint32_t w[8];
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        bf16 e[2];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const int i = 2 * h + k, n = n0 + c0 + i;
                            if (EPI == kEpiBf16Relu) {
                                e[k] = __float2bfloat16_rn(fmaxf(v[i] + g.bias[n], 0.0f));
                            } else {
                                e[k] = __float2bfloat16_rn(ar[i] > 0.0f ? v[i] : 0.0f);
                            }
                            if (g.OT) g.OT[(size_t)n * g.ldot + row] = e[k];
                        }
                        w[h] = (uint32_t)__bfloat16_as_ushort(e[0]) | ((uint32_t)__bfloat16_as_ushort(e[1]) << 16);
                    }
                    uint4* op = reinterpret_cast<uint4*>(g.O + (size_t)row * g.ldo + n0 + c0);
                    op[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    op[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    continue;
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + c0 + i;
                if (n >= g.N) continue;
                if (EPI == kEpiF32) {
                    g.C[(size_t)row * g.ldc + n] = v[i] + (g.bias ? g.bias[n] : 0.0f);
                } else if (EPI == kEpiPartial) {
                    g.C[(size_t)blockIdx.z * g.split_stride + (size_t)row * g.ldc + n] = v[i];
                } else if (EPI == kEpiBf16Relu) {
                    const bf16 h = __float2bfloat16_rn(fmaxf(v[i] + g.bias[n], 0.0f));
                    g.O[(size_t)row * g.ldo + n] = h;
                    if (g.OT) g.OT[(size_t)n * g.ldot + row] = h;
                } else {  // kEpiReluGrad
                    const float a = __bfloat162float(g.act[(size_t)row * g.ldact + n]);
                    const bf16 d = __float2bfloat16_rn(a > 0.0f ? v[i] : 0.0f);
                    g.O[(size_t)row * g.ldo + n] = d;
                    if (g.OT) g.OT[(size_t)n * g.ldot + row] = d;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// input features of sample i (origin ray r of bin i when origin_ray is given);
// zero for i >= n or an empty bin
__device__ __forceinline__ void mlp_features(const float* __restrict__ pos, const float* __restrict__ nrm,
                                             const uint32_t* __restrict__ origin_ray, uint32_t i, uint32_t n,
                                             float lox, float loy, float loz, float inv_s, float f[kIn]) {
#pragma unroll
    for (int k = 0; k < kIn; ++k) f[k] = 0.0f;
    const uint32_t r = origin_ray ? (i < n ? origin_ray[i] : kNone) : i;
    if (i < n && r != kNone) {
        const float ph[3] = {(pos[3 * (size_t)r + 0] - lox) * inv_s, (pos[3 * (size_t)r + 1] - loy) * inv_s,
                             (pos[3 * (size_t)r + 2] - loz) * inv_s};
        f[0] = ph[0];
        f[1] = ph[1];
        f[2] = ph[2];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float sc = (float)(1 << k);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                f[3 + 6 * k + a] = sinpif(sc * ph[a]);
                f[6 + 6 * k + a] = cospif(sc * ph[a]);
            }
        }
        f[75] = nrm[3 * (size_t)r + 0];
        f[76] = nrm[3 * (size_t)r + 1];
        f[77] = nrm[3 * (size_t)r + 2];
    }
}

// ---------------------------------------------------------------------------
// The three hidden layers, fused per 128-row tile: each thread computes the
// input features of its row into shared memory (bfloat16, the MMA's K-major
// layout), then every layer is one MMA into tensor memory (K = 80, then 64)
// whose epilogue (bias, ReLU, bfloat16) writes the activations back over the
// same shared tile for the next layer and out to global memory: row-major H3
// always, H1 and H2 and the transposes X^T, H1^T, H2^T, H3^T when given (a
// training step's weight gradients and ReLU masks).  128 threads, thread =
// row = TMEM lane; 64 TMEM columns; four CTAs per SM.
constexpr int kHidThreads = 128;
constexpr int kHidSmemX = 0, kHidSmemW1 = 20480, kHidSmemW2 = 30720, kHidSmemW3 = 38912, kHidSmemB = 47104;
constexpr int kHidSmemBytes = kHidSmemB + 3 * kHid * 4;

struct HiddenArgs {
    const float* pos;
    const float* nrm;
    const uint32_t* origin_ray;  // bins' origin rays, or null (row i = sample i)
    const uint32_t* n_dev;       // device row count (<= n_cap), or null (n_cap rows)
    uint32_t n_cap;
    float lo[3], inv_s;
    const bf16 *w1, *w2, *w3;    // [64][80], [64][64], [64][64]
    const float *b1, *b2, *b3;
    bf16 *h1, *h2, *h3;          // [rows][64]; h1, h2 may be null
    bf16 *xt, *h1t, *h2t, *h3t;  // [80][ldt] (rows 0..79 of X^T; row 78 = 1), [64 of 80][ldt]; null: not written
    int ldt;
    uint32_t* status;
};

__global__ void __launch_bounds__(kHidThreads, 4) k_mlp_hidden(HiddenArgs a) {
    extern __shared__ __align__(1024) uint8_t hid_smem[];
    uint8_t* sX = hid_smem + kHidSmemX;  // X tile 128 x 80 (K = 80), then H1, H2: 128 x 64 (K = 64)
    float* sb = reinterpret_cast<float*>(hid_smem + kHidSmemB);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t i = blockIdx.x * 128 + tid;  // row of this thread
    const bool in = i < a.n_cap;
    if (warp == 0) tc::tmem_alloc(&tmem_base, 64);
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    load_tile_async<kIn, kHidThreads>(hid_smem + kHidSmemW1, a.w1, kIn, 0, kHid, kHid, 0, kIn);
    load_tile_async<kHid, kHidThreads>(hid_smem + kHidSmemW2, a.w2, kHid, 0, kHid, kHid, 0, kHid);
    load_tile_async<kHid, kHidThreads>(hid_smem + kHidSmemW3, a.w3, kHid, 0, kHid, kHid, 0, kHid);
    tc::cp_async_commit();
    for (int j = tid; j < 3 * kHid; j += kHidThreads) sb[j] = (j < kHid ? a.b1 : j < 2 * kHid ? a.b2 : a.b3)[j % kHid];
    {
        const uint32_t n = a.n_dev ? min(*a.n_dev, a.n_cap) : a.n_cap;
        float f[kIn];
        mlp_features(a.pos, a.nrm, a.origin_ray, i, n, a.lo[0], a.lo[1], a.lo[2], a.inv_s, f);
#pragma unroll
        for (int q = 0; q < kIn / 8; ++q) {  // one 16-byte core-matrix row per 8 features
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 p = __floats2bfloat162_rn(f[8 * q + 2 * h], f[8 * q + 2 * h + 1]);
                w[h] = *reinterpret_cast<const uint32_t*>(&p);
            }
            *reinterpret_cast<uint4*>(sX + cm_off<kIn>(tid, 8 * q)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (a.xt && in) {  // consecutive threads write consecutive entries of each row of X^T
#pragma unroll
            for (int k = 0; k < kIn; ++k) a.xt[(size_t)k * a.ldt + i] = __float2bfloat16_rn(k == kFeatIn ? 1.0f : f[k]);
        }
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base, lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kHid);
    bool ok = true;
    uint32_t phase = 0;
#pragma unroll 1
    for (int l = 0; l < 3 && ok; ++l) {
        if (tid == 0) {
            const int K = l == 0 ? kIn : kHid;
            const uint32_t a0 = tc::smem_addr(sX),
                           b0 = tc::smem_addr(hid_smem + (l == 0 ? kHidSmemW1 : l == 1 ? kHidSmemW2 : kHidSmemW3));
            for (int k = 0; k < K / 16; ++k)
                tc::mma_bf16(tmem, tc::smem_desc(a0 + k * 256, 128, K * 16), tc::smem_desc(b0 + k * 256, 128, K * 16),
                             idesc, k > 0 ? 1u : 0u);
            tc::mma_commit(&mbar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&mbar, phase)) != 0;
        phase ^= 1u;
        tc::fence_after_sync();
        if (!ok) break;
        bf16* O = l == 0 ? a.h1 : l == 1 ? a.h2 : a.h3;
        bf16* OT = l == 0 ? a.h1t : l == 1 ? a.h2t : a.h3t;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_base + (uint32_t)c0, v);
            uint32_t w[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const __nv_bfloat162 p = __floats2bfloat162_rn(fmaxf(v[2 * h] + sb[l * kHid + c0 + 2 * h], 0.0f),
                                                               fmaxf(v[2 * h + 1] + sb[l * kHid + c0 + 2 * h + 1], 0.0f));
                w[h] = *reinterpret_cast<const uint32_t*>(&p);
            }
            if (l < 2) {  // the next layer's A operand (the MMA of this layer has completed)
                *reinterpret_cast<uint4*>(sX + cm_off<kHid>(tid, c0)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(sX + cm_off<kHid>(tid, c0 + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
            }
            if (O && in) {
                uint4* op = reinterpret_cast<uint4*>(O + (size_t)i * kHid + c0);
                op[0] = make_uint4(w[0], w[1], w[2], w[3]);
                op[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
            if (OT && in) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    OT[(size_t)(c0 + j) * a.ldt + i] =
                        __ushort_as_bfloat16((unsigned short)((w[j >> 1] >> (16 * (j & 1))) & 0xffffu));
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();  // the accumulator has been read; the next layer's A tile is staged
        tc::fence_after_sync();
    }
    if (!ok && (tid & 31) == 0) atomicOr(a.status, (uint32_t)WFPG_STATUS_MMA_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// The sum over the K splits of a [M][ncols] weight-and-bias gradient (a block
// covers 32 outputs, its 8 warps take every 8th split, the 8 partial sums are
// added in warp order: deterministic): column c < wcols of row m goes to
// out_w[m * ldw + c], column bias_col to out_b[m], the rest is dropped
__global__ void __launch_bounds__(256) k_sum_splits_wb(const float* __restrict__ part, int splits, uint32_t mn,
                                                       int ncols, float* __restrict__ out_w, int ldw, int wcols,
                                                       float* __restrict__ out_b, int bias_col) {
    __shared__ float red[8][32];
    const uint32_t i = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.0f;
    if (i < mn)
        for (int z = threadIdx.y; z < splits; z += 8) acc += part[(size_t)z * mn + i];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && i < mn) {
        float sum = 0.0f;
#pragma unroll
        for (int y = 0; y < 8; ++y) sum += red[y][threadIdx.x];
        const uint32_t m = i / (uint32_t)ncols, c = i % (uint32_t)ncols;
        if ((int)c < wcols) out_w[(size_t)m * ldw + c] = sum;
        else if ((int)c == bias_col) out_b[m] = sum;
    }
}

// out[i] = v for i < n (bfloat16)
__global__ void k_fill_bf16(bf16* __restrict__ out, uint32_t n, float v) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// The output layer of a training step, fused: for one 128-row tile, the logits
// Z = H3 W4^T + b4 (1024 per row) are computed 64 at a time on the tensor
// cores into tensor memory and never stored.  Pass 1 keeps each row's running
// maximum and exponential sum (base 2: u = Z log2 e) and the sums T = sum t
// and A = sum t log2 t of its target row t; pass 2 recomputes each chunk,
// forms the logit gradient G = bf16((softmax(Z) - t / T) / n), stores G^T
// (the weight-gradient GEMM dW4 = G^T [H3 | 1] gives dW4 and db4) and
// accumulates dA3 = G W4 in tensor memory with a second MMA per chunk.  The
// KL term of a row needs no per-element logarithm of q: with S the base-2 log
// of the softmax denominator and B = sum t u,
//   KL = sum q (ln q - ln p) = ln 2 (A / T - log2 T - B / T + S)   (T > 0).
// The epilogue writes d3 = bf16(dA3 o [H3 > 0]) and its transpose.  256
// threads, four CTAs per SM (128 TMEM columns each): warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (the tile's rows) and handles columns 32 (w / 4) .. + 31
// of each chunk.  Pass 1 double-buffers the logits (TMEM columns 0 and 64)
// and the W4 rows (the W4^T buffer is free then); in pass 2 the dA3 MMA of a
// chunk and the logits MMA of the next one are issued together.  Rows past n
// take zero weight and write zeros (the transposes are mpad >= 128 ceil(n /
// 128) rows long).
constexpr int kOutThreads = 256;
constexpr int kOutChunk = 64;                  // logits per chunk
constexpr int kOutChunks = kOut / kOutChunk;   // 16
constexpr uint32_t kOutTmemCols = 128;
constexpr int kOutSmemH = 0, kOutSmemW = 16384, kOutSmemWT = 24576, kOutSmemG = 32768, kOutSmemB = 49152;
constexpr int kOutSmemBytes = kOutSmemB + 4 * kOut;
constexpr float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;

struct OutTrainArgs {
    const bf16* h3;      // [n][64]
    const bf16* w4;      // [1024][64]
    const bf16* w4t;     // [64][1024]
    const float* b4;     // [1024]
    const float* target; // [n][1024], any non-negative field per row (normalised here); 32-byte aligned
    int n;
    float inv_n;
    bf16* g4t;           // [1024][ldg]: G^T
    int ldg;
    bf16* d3;            // [ldg][64]
    bf16* d3t;           // [64][ldg]
    float* loss;         // accumulated mean KL
    uint32_t* status;
};

// base-2 exponential and logarithm of the special function unit
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// eight floats with one 32-byte load that bypasses L1 (p 32-byte aligned)
__device__ __forceinline__ void ld8_stream(const float* p, float v[8]) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}

__global__ void __launch_bounds__(kOutThreads, 4)
    k_out_train(const __grid_constant__ CUtensorMap tma_h3, const __grid_constant__ CUtensorMap tma_w4,
                const __grid_constant__ CUtensorMap tma_w4t, OutTrainArgs a) {
    extern __shared__ __align__(1024) uint8_t out_smem_raw[];
    // the TMA tiles (128-byte swizzled) need 1024-byte alignment (the launch adds 1 KB of slack)
    uint8_t* out_smem = out_smem_raw + ((1024u - (tc::smem_addr(out_smem_raw) & 1023u)) & 1023u);
    uint8_t* sH = out_smem + kOutSmemH;    // H3 tile: 128 x 64 (K = 64), TMA, 128-byte swizzled
    uint8_t* sW = out_smem + kOutSmemW;    // W4 rows of the chunk: 64 x 64, TMA, swizzled
    uint8_t* sWT = out_smem + kOutSmemWT;  // W4^T columns of the chunk (pass 2) / second W4 buffer (pass 1)
    uint8_t* sG = out_smem + kOutSmemG;    // G of the chunk: 128 x 64, core matrices; row statistics after pass 1
    float* sbl = reinterpret_cast<float*>(out_smem + kOutSmemB);  // b4 log2 e
    __shared__ __align__(8) uint64_t mbar[2];  // MMA completion: logits buffer 0 / 1
    __shared__ __align__(8) uint64_t tbar[3];  // TMA completion: sW, sWT, sH
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int r = quad * 32 + lane;  // tile row of this thread
    const int m0 = blockIdx.x * 128, row = m0 + r;
    const bool live = row < a.n;
    const int k0 = half * 32;        // first chunk column of this thread
    const int rot = blockIdx.x & (kOutChunks - 1);  // chunk order rotated by CTA: spreads the target reads
    auto chunk = [rot](int c) { return (c + rot) & (kOutChunks - 1); };
    // thread 0 issues every TMA copy and MMA; tph holds the parity of each TMA barrier's
    // next phase, tpend the barriers with a copy in flight, tok whether its waits succeeded
    uint32_t tph = 0, tpend = 0;
    bool tok = true;
    auto tma_w = [&](uint8_t* dst, int bi, int c) {  // W4 rows of chunk c (x = 0)
        tc::mbar_expect_tx(&tbar[bi], 64 * 64 * 2);
        tc::tma_load_2d(dst, &tma_w4, 0, c * kOutChunk, &tbar[bi]);
        tpend |= 1u << bi;
    };
    auto tma_wt = [&](int c) {  // W4^T columns of chunk c (x = 64 c: 128-byte aligned)
        tc::mbar_expect_tx(&tbar[1], 64 * 64 * 2);
        tc::tma_load_2d(sWT, &tma_w4t, c * kOutChunk, 0, &tbar[1]);
        tpend |= 1u << 1;
    };
    auto tma_done = [&](int bi) {
        tok = tc::mbar_wait(&tbar[bi], (tph >> bi) & 1u) && tok;
        tph ^= 1u << bi;
        tpend &= ~(1u << bi);
    };
    if (warp == 0) tc::tmem_alloc(&tmem_base, kOutTmemCols);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        for (int i = 0; i < 3; ++i) tc::mbar_init(&tbar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tc::mbar_expect_tx(&tbar[2], 128 * 64 * 2);
        tc::tma_load_2d(sH, &tma_h3, 0, m0, &tbar[2]);  // rows past n read zero
        tpend |= 1u << 2;
        tma_w(sW, 0, chunk(0));
        tma_w(sWT, 1, chunk(1));
    }
    for (int i = tid; i < kOut; i += kOutThreads) sbl[i] = a.b4[i] * kLog2e;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);  // every MMA: M = 128, N = 64, K = 64
    const float* trow = a.target + (size_t)(live ? row : a.n - 1) * kOut;
    uint32_t phase = 0;  // bit i: parity of mbar[i]'s next phase
    bool ok = true;
    // D (+)= A B^T over K = 64 as four K = 16 MMAs (issued by thread 0 only); B is a
    // swizzled TMA tile, A either the swizzled H3 tile (the logits) or the core-matrix G tile (dA3)
    auto mma64 = [&](uint32_t d, const uint8_t* A, bool a_swizzled, const uint8_t* B, bool acc) {
        const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
#pragma unroll
        for (int s = 0; s < 4; ++s)
            tc::mma_bf16(d, a_swizzled ? tc::smem_desc_sw128(a0 + s * 32) : tc::smem_desc(a0 + s * 256, 128, 64 * 16),
                         tc::smem_desc_sw128(b0 + s * 32), idesc, (acc || s > 0) ? 1u : 0u);
    };
    auto wait_bar = [&](int i) {
        ok = ok && __syncthreads_and(tc::mbar_wait(&mbar[i], (phase >> i) & 1u) && tok) != 0;
        phase ^= 1u << i;
        tc::fence_after_sync();
    };
    if (tid == 0) {
        tma_done(2);
        tma_done(0);
        mma64(tmem, sH, true, sW, false);
        tc::mma_commit(&mbar[0]);
        tma_done(1);
        mma64(tmem + 64, sH, true, sWT, false);
        tc::mma_commit(&mbar[1]);
    }

    // ---- pass 1: running maximum and base-2 exponential sum of this thread's columns; T and A of the target row
    float mrun = -3.0e38f, srun = 0.0f;
    float* s_st = reinterpret_cast<float*>(sG);  // [m, s][2 column halves][128 rows], then T[128], A[128]
    for (int c = 0; c < kOutChunks && ok; ++c) {
        const int buf = c & 1;
        // the target sums of one whole row per warp and chunk (tile row 16 warp + c), read contiguously
        const int lr = warp * 16 + c;
        const float* tr = a.target + (size_t)min(m0 + lr, a.n - 1) * kOut + lane * 8;
        float t[32];
#pragma unroll
        for (int i = 0; i < 4; ++i) ld8_stream(tr + 256 * i, t + 8 * i);
        wait_bar(buf);
        if (!ok) break;
        if (tid == 0 && c + 2 < kOutChunks) tma_w(buf ? sWT : sW, buf, chunk(c + 2));  // the MMA has read the buffer
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float v[16];
            tc::tmem_ld16(lane_base + (uint32_t)(64 * buf + k0 + g * 16), v);
            const float4* bq = reinterpret_cast<const float4*>(sbl + chunk(c) * kOutChunk + k0 + g * 16);
            float gm = -3.0e38f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 b = bq[i];
                v[4 * i + 0] = fmaf(v[4 * i + 0], kLog2e, b.x);
                v[4 * i + 1] = fmaf(v[4 * i + 1], kLog2e, b.y);
                v[4 * i + 2] = fmaf(v[4 * i + 2], kLog2e, b.z);
                v[4 * i + 3] = fmaf(v[4 * i + 3], kLog2e, b.w);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) gm = fmaxf(gm, v[i]);
            if (gm > mrun) {
                srun *= ex2_approx(mrun - gm);
                mrun = gm;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) srun += ex2_approx(v[i] - mrun);
        }
        float tsum = 0.0f, tlog = 0.0f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            tsum += t[i];
            tlog = fmaf(t[i], lg2_approx(fmaxf(t[i], 1e-30f)), tlog);  // t = 0 adds 0
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
            tlog += __shfl_xor_sync(0xffffffffu, tlog, o);
        }
        if (lane == 0) {
            s_st[512 + lr] = tsum;
            s_st[640 + lr] = tlog;
        }
        tc::fence_before_sync();
        __syncthreads();  // the logits have been read
        tc::fence_after_sync();
        if (tid == 0 && c + 2 < kOutChunks) {
            tma_done(buf);  // the W4 rows of chunk c + 2
            mma64(tmem + 64 * buf, sH, true, buf ? sWT : sW, false);
            tc::mma_commit(&mbar[buf]);
        }
    }
    s_st[0 * 256 + half * 128 + r] = mrun;
    s_st[1 * 256 + half * 128 + r] = srun;
    if (tid == 0 && ok) {  // pass 2 starts at the last chunk (both buffers' MMAs are done)
        tma_w(sW, 0, chunk(kOutChunks - 1));
        tma_wt(chunk(kOutChunks - 1));
    }
    __syncthreads();
    float S, invT, A, tsum;
    {
        const float ma = s_st[r], mb = s_st[128 + r];
        const float m = fmaxf(ma, mb);
        S = m + lg2_approx(s_st[256 + r] * ex2_approx(ma - m) + s_st[384 + r] * ex2_approx(mb - m));
        tsum = s_st[512 + r];
        A = s_st[640 + r];
        invT = tsum > 0.0f ? 1.0f / tsum : 0.0f;
    }
    // G = p / n - t / (T n); rows past n give zero
    const float gp = live ? a.inv_n : 0.0f, gq = live ? -invT * a.inv_n : 0.0f;
    float bsum = 0.0f;  // B = sum t u over this thread's columns
    tc::fence_before_sync();
    __syncthreads();  // the statistics have been read (sG is G again)
    tc::fence_after_sync();
    if (tid == 0 && ok) {
        tma_done(0);
        mma64(tmem, sH, true, sW, false);
        tc::mma_commit(&mbar[0]);
    }

    // ---- pass 2, chunks in reverse (the target rows read last are read again first)
    for (int i = 0; i < kOutChunks && ok; ++i) {
        const int c = chunk(kOutChunks - 1 - i);
        float t[32];
#pragma unroll
        for (int k = 0; k < 4; ++k) ld8_stream(trow + c * kOutChunk + k0 + 8 * k, t + 8 * k);
        wait_bar(0);  // the logits of chunk c are in TMEM; the previous dA3 MMA has read sG and W4^T
        if (!ok) break;
        if (tid == 0) {  // the logits MMA has read sW, the last dA3 MMA sWT
            if (i > 0) tma_wt(c);
            if (i + 1 < kOutChunks) tma_w(sW, 0, chunk(kOutChunks - 2 - i));
        }
        bf16* gcol = a.g4t + (size_t)(c * kOutChunk + k0) * a.ldg + row;  // G^T of this thread's first column
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float v[16];
            tc::tmem_ld16(lane_base + (uint32_t)(k0 + g * 16), v);
            const float4* bq = reinterpret_cast<const float4*>(sbl + c * kOutChunk + k0 + g * 16);
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // 8 columns: one 16-byte row of a core matrix
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float4 b = bq[2 * h + e];
                    const float bb[4] = {b.x, b.y, b.z, b.w};
                    float gv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int j = 8 * h + 4 * e + k;
                        const float u = fmaf(v[j], kLog2e, bb[k]);
                        const float tj = t[g * 16 + j];
                        bsum = fmaf(tj, u, bsum);
                        gv[k] = fmaf(ex2_approx(u - S), gp, tj * gq);
                    }
                    const __nv_bfloat162 lo = __floats2bfloat162_rn(gv[0], gv[1]);
                    const __nv_bfloat162 hi = __floats2bfloat162_rn(gv[2], gv[3]);
                    w[2 * e] = *reinterpret_cast<const uint32_t*>(&lo);
                    w[2 * e + 1] = *reinterpret_cast<const uint32_t*>(&hi);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t x = (w[j >> 1] >> (16 * (j & 1))) & 0xffffu;
                    gcol[(size_t)(g * 16 + 8 * h + j) * a.ldg] = __ushort_as_bfloat16((unsigned short)x);
                }
                *reinterpret_cast<uint4*>(sG + cm_off<64>(r, k0 + g * 16 + 8 * h)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_proxy_async();  // G, written by the threads, is read by the tensor cores
        tc::fence_before_sync();
        __syncthreads();  // G staged, the logits read
        tc::fence_after_sync();
        if (tid == 0) {
            tma_done(1);  // W4^T of chunk c
            mma64(tmem + (uint32_t)kOutChunk, sG, false, sWT, i > 0);
            if (i + 1 < kOutChunks) {
                tma_done(0);  // W4 of the next chunk
                mma64(tmem, sH, true, sW, false);
            }
            tc::mma_commit(&mbar[0]);
        }
    }
    if (ok) wait_bar(0);  // the last dA3 MMA
    if (tid == 0) {  // after a timeout, let the copies in flight land before the CTA exits
        for (int bi = 0; bi < 3; ++bi)
            if (tpend & (1u << bi)) tma_done(bi);
    }
    if (!ok && lane == 0) atomicOr(a.status, (uint32_t)WFPG_STATUS_MMA_TIMEOUT);
    // every thread reads the H3 tile below: observe its copy's completion (phase 0)
    const bool h3_ok = tc::mbar_wait(&tbar[2], 0u);

    // ---- epilogue: d3 = bf16(dA3 o [H3 > 0]) (this thread's 32 of the 64 columns) and its transpose; the KL
    if (ok && h3_ok) {
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            float v[16];
            tc::tmem_ld16(lane_base + (uint32_t)(kOutChunk + half * 32 + g * 16), v);
            uint32_t w[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                bf16 x[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int j = half * 32 + g * 16 + 2 * h + k;
                    // element (r, j) of the swizzled tile: 16-byte chunk j / 8 of row r at chunk (j / 8) ^ (r % 8)
                    const float hv = __bfloat162float(*reinterpret_cast<const bf16*>(
                        sH + (r >> 3) * 1024 + (r & 7) * 128 + ((((j >> 3) ^ r) & 7) << 4) + (j & 7) * 2));
                    x[k] = __float2bfloat16_rn(hv > 0.0f ? v[2 * h + k] : 0.0f);
                    a.d3t[(size_t)j * a.ldg + row] = x[k];
                }
                w[h] = (uint32_t)__bfloat16_as_ushort(x[0]) | ((uint32_t)__bfloat16_as_ushort(x[1]) << 16);
            }
            uint4* dp = reinterpret_cast<uint4*>(a.d3 + (size_t)row * kHid + half * 32 + g * 16);
            dp[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dp[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
        float kl = 0.0f;
        if (live && tsum > 0.0f)
            kl = kLn2 * ((half == 0 ? A * invT - lg2_approx(tsum) + S : 0.0f) - bsum * invT);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kl += __shfl_xor_sync(0xffffffffu, kl, o);
        if (lane == 0) atomicAdd(a.loss, kl * a.inv_n);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kOutTmemCols);
}

// ---------------------------------------------------------------------------
// The output layer of an inference, fused: for one 128-row tile the logits
// Z = H3 W4^T + b4 are computed 64 at a time on the tensor cores into tensor
// memory and never stored.  Pass 1 keeps each row's running maximum and base-2
// exponential sum (u = Z log2 e); pass 2 recomputes every chunk and writes the
// field softmax(Z) + eps = 2^(u - S) + eps, S the base-2 log of the softmax
// denominator.  The logits MMAs of both passes run as one pipeline of 32 chunks,
// double-buffered in TMEM (columns 0 and 64) and in shared memory (two W4 row
// blocks by TMA).  256 threads, four CTAs per SM: warp w reads TMEM lanes
// 32 (w % 4) .. + 31 and handles columns 32 (w / 4) .. + 31 of each chunk.
constexpr int kInferSmemH = 0, kInferSmemW0 = 16384, kInferSmemW1 = 24576, kInferSmemB = 32768,
              kInferSmemStat = kInferSmemB + 4 * kOut;
constexpr int kInferSmemBytes = kInferSmemStat + 2 * 2 * 128 * 4;

struct InferArgs {
    const float* b4;   // [1024]
    int n;             // rows
    float eps;
    float* field;      // [n][1024]: softmax + eps
    uint32_t* status;
};

__global__ void __launch_bounds__(kOutThreads, 4)
    k_out_infer(const __grid_constant__ CUtensorMap tma_h3, const __grid_constant__ CUtensorMap tma_w4, InferArgs a) {
    extern __shared__ __align__(1024) uint8_t inf_smem_raw[];
    // the TMA tiles (128-byte swizzled) need 1024-byte alignment (the launch adds 1 KB of slack)
    uint8_t* sm = inf_smem_raw + ((1024u - (tc::smem_addr(inf_smem_raw) & 1023u)) & 1023u);
    uint8_t* sH = sm + kInferSmemH;                       // H3 tile: 128 x 64
    auto sW = [sm](int b) { return sm + (b ? kInferSmemW1 : kInferSmemW0); };  // W4 rows for logits buffer b
    float* sbl = reinterpret_cast<float*>(sm + kInferSmemB);    // b4 log2 e
    float* s_st = reinterpret_cast<float*>(sm + kInferSmemStat);  // [m, s][2 column halves][128 rows]
    __shared__ __align__(8) uint64_t mbar[2];  // MMA completion: logits buffer 0 / 1
    __shared__ __align__(8) uint64_t tbar[3];  // TMA completion: W4 buffer 0 / 1, H3
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int r = quad * 32 + lane;  // tile row of this thread
    const int m0 = blockIdx.x * 128, row = m0 + r;
    const int k0 = half * 32;
    constexpr int kSteps = 2 * kOutChunks;  // pass 1 then pass 2, chunk it % 16
    uint32_t tph = 0, tpend = 0;            // thread 0: parity of each TMA barrier's next phase, copies in flight
    bool tok = true;
    auto tma_w = [&](int bi, int c) {
        tc::mbar_expect_tx(&tbar[bi], 64 * 64 * 2);
        tc::tma_load_2d(sW(bi), &tma_w4, 0, c * kOutChunk, &tbar[bi]);
        tpend |= 1u << bi;
    };
    auto tma_done = [&](int bi) {
        tok = tc::mbar_wait(&tbar[bi], (tph >> bi) & 1u) && tok;
        tph ^= 1u << bi;
        tpend &= ~(1u << bi);
    };
    if (warp == 0) tc::tmem_alloc(&tmem_base, kOutTmemCols);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        for (int i = 0; i < 3; ++i) tc::mbar_init(&tbar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tc::mbar_expect_tx(&tbar[2], 128 * 64 * 2);
        tc::tma_load_2d(sH, &tma_h3, 0, m0, &tbar[2]);  // rows past n read zero
        tpend |= 1u << 2;
        tma_w(0, 0);
        tma_w(1, 1);
    }
    for (int i = tid; i < kOut; i += kOutThreads) sbl[i] = a.b4[i] * kLog2e;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);
    auto mma_z = [&](int buf) {  // logits of the chunk in W4 buffer buf into TMEM columns 64 buf
        const uint32_t a0 = tc::smem_addr(sH), b0 = tc::smem_addr(sW(buf));
#pragma unroll
        for (int s = 0; s < 4; ++s)
            tc::mma_bf16(tmem + 64 * buf, tc::smem_desc_sw128(a0 + s * 32), tc::smem_desc_sw128(b0 + s * 32), idesc,
                         s > 0 ? 1u : 0u);
        tc::mma_commit(&mbar[buf]);
    };
    if (tid == 0) {
        tma_done(2);
        tma_done(0);
        mma_z(0);
        tma_done(1);
        mma_z(1);
    }
    uint32_t phase = 0;  // bit i: parity of mbar[i]'s next phase
    bool ok = true;
    float mrun = -3.0e38f, srun = 0.0f, S = 0.0f;
    const bool live = row < a.n;
    for (int it = 0; it < kSteps && ok; ++it) {
        const int buf = it & 1, c = it % kOutChunks;
        ok = __syncthreads_and(tc::mbar_wait(&mbar[buf], (phase >> buf) & 1u) && tok) != 0;
        phase ^= 1u << buf;
        tc::fence_after_sync();
        if (!ok) break;
        if (tid == 0 && it + 2 < kSteps) tma_w(buf, (it + 2) % kOutChunks);  // the MMA has read the buffer
        if (it == kOutChunks) {  // both halves' statistics were exchanged at the end of pass 1
            const float ma = s_st[r], mb = s_st[128 + r];
            const float m = fmaxf(ma, mb);
            S = m + lg2_approx(s_st[256 + r] * ex2_approx(ma - m) + s_st[384 + r] * ex2_approx(mb - m));
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float v[16];
            tc::tmem_ld16(lane_base + (uint32_t)(64 * buf + k0 + g * 16), v);
            const float4* bq = reinterpret_cast<const float4*>(sbl + c * kOutChunk + k0 + g * 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 b = bq[i];
                v[4 * i + 0] = fmaf(v[4 * i + 0], kLog2e, b.x);
                v[4 * i + 1] = fmaf(v[4 * i + 1], kLog2e, b.y);
                v[4 * i + 2] = fmaf(v[4 * i + 2], kLog2e, b.z);
                v[4 * i + 3] = fmaf(v[4 * i + 3], kLog2e, b.w);
            }
            if (it < kOutChunks) {
                float gm = -3.0e38f;
#pragma unroll
                for (int i = 0; i < 16; ++i) gm = fmaxf(gm, v[i]);
                if (gm > mrun) {
                    srun *= ex2_approx(mrun - gm);
                    mrun = gm;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) srun += ex2_approx(v[i] - mrun);
            } else if (live) {
                float4* fp = reinterpret_cast<float4*>(a.field + (size_t)row * kOut + c * kOutChunk + k0 + g * 16);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    fp[i] = make_float4(ex2_approx(v[4 * i] - S) + a.eps, ex2_approx(v[4 * i + 1] - S) + a.eps,
                                        ex2_approx(v[4 * i + 2] - S) + a.eps, ex2_approx(v[4 * i + 3] - S) + a.eps);
            }
        }
        if (it == kOutChunks - 1) {
            s_st[half * 128 + r] = mrun;
            s_st[256 + half * 128 + r] = srun;
        }
        tc::fence_before_sync();
        __syncthreads();  // the logits have been read (and the statistics exchanged)
        tc::fence_after_sync();
        if (tid == 0 && it + 2 < kSteps) {
            tma_done(buf);  // the W4 rows of step it + 2
            mma_z(buf);
        }
    }
    if (tid == 0) {  // after a timeout, let the copies in flight land before the CTA exits
        for (int bi = 0; bi < 3; ++bi)
            if (tpend & (1u << bi)) tma_done(bi);
    }
    if (!ok && lane == 0) atomicOr(a.status, (uint32_t)WFPG_STATUS_MMA_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kOutTmemCols);
}

// Adam (Kingma & Ba 2015) on the float32 master weights
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, uint32_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 copies of the weights: W[out][in] and its transpose
__global__ void k_convert(const float* __restrict__ W, int nout, int nin, bf16* __restrict__ Wb,
                          bf16* __restrict__ WbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nout * nin) return;
    const int o = i / nin, k = i % nin;
    const bf16 b = __float2bfloat16_rn(W[i]);
    Wb[i] = b;
    if (WbT) WbT[(size_t)k * nout + o] = b;
}

}  // namespace

struct wfpg_mlp {
    int device = 0;
    uint32_t max_batch = 0, mpad = 0;
    uint32_t ldt = 0;  // row stride of the transposed activations: mpad + 64, off the power-of-two strides
    int step = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    bf16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *w4 = nullptr, *w2t = nullptr, *w3t = nullptr,
         *w4t = nullptr;
    bf16 *xt = nullptr, *h1 = nullptr, *h1t = nullptr, *h2 = nullptr, *h2t = nullptr, *h3 = nullptr,
         *h3t = nullptr, *g4t = nullptr, *d3 = nullptr, *d3t = nullptr, *d2 = nullptr,
         *d2t = nullptr, *d1 = nullptr, *d1t = nullptr;
    float* z = nullptr;
    float* part = nullptr;  // split-K partial weight gradients
    float* field = nullptr;
    float* loss = nullptr;
    uint32_t* status = nullptr;
};

namespace {

// launches the GEMM; returns the number of K splits it used
// cuTensorMapEncodeTiled of the driver, fetched once through the runtime (no link
// dependency on the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// 2-D tensor map of a bf16 matrix [rows][ld] whose first K entries per row are used:
// boxes of 64 (K) x box_rows, 128-byte swizzling, zero fill outside; false when the
// driver refuses it
bool tensor_map(CUtensorMap* m, const bf16* base, int K, int rows, int ld, int box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || K < 1 || rows < 1) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t stride[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estride[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dim, stride, box, estride,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// set when a GEMM could not be launched (its tensor maps were refused); read and
// cleared by the entry points
thread_local bool g_gemm_failed = false;
bool gemm_failed() {
    const bool f = g_gemm_failed;
    g_gemm_failed = false;
    return f;
}

template <int BN, int EPI>
int gemm(const GemmArgs& a, int splits, cudaStream_t st) {
    constexpr int kKChunk = KChunk<BN>::value;
    GemmArgs g = a;
    const int chunks = (g.K + kKChunk - 1) / kKChunk;
    if (splits < 1) splits = 1;
    if (splits > chunks) splits = chunks;
    g.chunks_per_split = (chunks + splits - 1) / splits;
    splits = (chunks + g.chunks_per_split - 1) / g.chunks_per_split;
    const dim3 grid(div_up(g.M, 128), div_up(g.N, BN), splits);
    auto kernel = k_gemm_tn<BN, EPI>;
    // up to kMaxStages tile stages, never more than a CTA's chunks (a single chunk
    // needs one: the smaller footprint keeps more CTAs resident), plus 1 KB so that
    // the kernel can align the swizzled tiles to 1024 bytes
    const int stage_bytes = (128 + BN) * kKChunk * 2;
    g.stages = std::max(1, std::min(kMaxStages, g.chunks_per_split));
    const int smem = g.stages * stage_bytes + 1024;
    static std::atomic<uint64_t> raised{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(raised.load(std::memory_order_relaxed) & bit)) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStages * stage_bytes + 1024);
        raised.fetch_or(bit, std::memory_order_relaxed);
    }
    alignas(64) CUtensorMap ta, tb;
    if (!tensor_map(&ta, g.A, g.K, g.M, g.lda, 128) || !tensor_map(&tb, g.B, g.K, g.N, g.ldb, BN)) {
        g_gemm_failed = true;
        return 0;
    }
    WFPG_LAUNCH(kernel, grid, kGemmThreads, smem, st, ta, tb, g);
    return splits;
}

// split-K weight and bias gradient: partial tiles [splits][M][kTRows] into s->part,
// then their sum: columns < wcols to out_w (row stride ldw), column bias_col to out_b
void weight_grad_wb(wfpg_mlp* s, GemmArgs g, float* out_w, int ldw, int wcols, float* out_b, int bias_col,
                    cudaStream_t st) {
    // one wave: a CTA per SM (four 53 KB stages each), the K range split over the SMs left per row tile
    const int splits = std::max(1, sm_count() / (int)div_up((uint64_t)g.M, 128));
    g.C = s->part;
    g.ldc = g.N;
    g.split_stride = (size_t)g.M * g.N;
    const int used = gemm<kTRows, kEpiPartial>(g, splits, st);
    if (used < 1) return;  // not launched: the entry point reports it
    const uint32_t mn = (uint32_t)(g.M * g.N);
    WFPG_LAUNCH(k_sum_splits_wb, div_up(mn, 32), dim3(32, 8), 0, st, s->part, used, mn, g.N, out_w, ldw, wcols,
                out_b, bias_col);
}

GemmArgs gargs(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, uint32_t* status) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.status = status;
    return g;
}

void convert_weights(wfpg_mlp* s, cudaStream_t st) {
    const int T = 256;
    WFPG_LAUNCH(k_convert, div_up(kHid * kIn, T), T, 0, st, s->params + kOffW1, kHid, kIn, s->w1, (bf16*)nullptr);
    WFPG_LAUNCH(k_convert, div_up(kHid * kHid, T), T, 0, st, s->params + kOffW2, kHid, kHid, s->w2, s->w2t);
    WFPG_LAUNCH(k_convert, div_up(kHid * kHid, T), T, 0, st, s->params + kOffW3, kHid, kHid, s->w3, s->w3t);
    WFPG_LAUNCH(k_convert, div_up(kOut * kHid, T), T, 0, st, s->params + kOffW4, kOut, kHid, s->w4, s->w4t);
}

// the hidden layers for n_cap rows (the row count is on the device when n_dev is
// given); a training step also keeps H1, H2 and the transposes
void hidden(wfpg_mlp* s, const float* pos, const float* nrm, const uint32_t* origin_ray, const uint32_t* n_dev,
            uint32_t n_cap, const wfpg_learned_params* p, bool training, cudaStream_t st) {
    HiddenArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pos = pos;
    a.nrm = nrm;
    a.origin_ray = origin_ray;
    a.n_dev = n_dev;
    a.n_cap = n_cap;
    for (int k = 0; k < 3; ++k) a.lo[k] = p->lo[k];
    a.inv_s = 1.0f / p->size;
    a.w1 = s->w1;
    a.w2 = s->w2;
    a.w3 = s->w3;
    a.b1 = s->params + kOffB1;
    a.b2 = s->params + kOffB2;
    a.b3 = s->params + kOffB3;
    a.h3 = s->h3;
    if (training) {
        a.h1 = s->h1;
        a.h2 = s->h2;
        a.xt = s->xt;
        a.h1t = s->h1t;
        a.h2t = s->h2t;
        a.h3t = s->h3t;
    }
    a.ldt = (int)s->ldt;
    a.status = s->status;
    WFPG_LAUNCH(k_mlp_hidden, div_up(n_cap, 128), kHidThreads, kHidSmemBytes, st, a);
}

// the logits Z = H3 W4^T + b4 of n rows into z_out ([n][1024]), else the handle's buffer
void output_logits(wfpg_mlp* s, int n, cudaStream_t st, float* z_out = nullptr) {
    GemmArgs g = gargs(s->h3, kHid, s->w4, kHid, n, kOut, kHid, s->status);
    g.C = z_out ? z_out : s->z;
    g.ldc = kOut;
    g.bias = s->params + kOffB4;
    gemm<256, kEpiF32>(g, 1, st);
}

int mlp_fail(int code, const std::string& msg) { return wfpg::set_last_error(code, msg); }

// one Adam step on the float32 master weights with the gradient `grad` (device,
// kParams floats), then fresh bfloat16 copies; the step count advances
void adam_update(wfpg_mlp* s, const float* grad, const wfpg_adam_params& opt, cudaStream_t st) {
    s->step += 1;
    const float c1 = 1.0f - powf(opt.beta1, (float)s->step), c2 = 1.0f - powf(opt.beta2, (float)s->step);
    WFPG_LAUNCH(k_adam, div_up(kParams, 256), 256, 0, st, s->params, s->m, s->v, grad, (uint32_t)kParams, opt.lr,
                opt.beta1, opt.beta2, opt.eps, c1, c2);
    convert_weights(s, st);
}

}  // namespace

namespace wfpg {
uint32_t mlp_max_batch(const wfpg_mlp* m) { return m->max_batch; }
}  // namespace wfpg

extern "C" {

int mlp_create(const float* params, uint32_t max_batch, void* stream, wfpg_mlp** out) {
    if (!out) return mlp_fail(WFPG_ERR_INVALID_ARG, "mlp_create: null out");
    *out = nullptr;
    if (max_batch == 0 || max_batch > (1u << 24))
        return mlp_fail(WFPG_ERR_INVALID_ARG, "mlp_create: max_batch must be in [1, 2^24]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wfpg_mlp* s = new wfpg_mlp();
    cudaGetDevice(&s->device);
    s->max_batch = max_batch;
    s->mpad = (max_batch + 127) / 128 * 128;
    s->ldt = s->mpad + 64;
    const size_t mp = s->mpad, lt = s->ldt;
    bool ok = true;
    auto alloc = [&](auto** p, size_t bytes) {
        if (ok && cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16) != cudaSuccess) ok = false;
    };
    alloc(&s->params, 4 * kParams);
    alloc(&s->m, 4 * kParams);
    alloc(&s->v, 4 * kParams);
    alloc(&s->grad, 4 * kParams);
    alloc(&s->part, 4 * (size_t)sm_count() * 128 * kTRows);  // splits x row tiles <= SMs, 128 rows each
    alloc(&s->w1, 2 * kHid * kIn);
    alloc(&s->w2, 2 * kHid * kHid);
    alloc(&s->w3, 2 * kHid * kHid);
    alloc(&s->w4, 2 * (size_t)kOut * kHid);
    alloc(&s->w2t, 2 * kHid * kHid);
    alloc(&s->w3t, 2 * kHid * kHid);
    alloc(&s->w4t, 2 * (size_t)kOut * kHid);
    alloc(&s->xt, 2 * lt * kIn);
    bf16** acts[] = {&s->h1, &s->h2, &s->h3, &s->d3, &s->d3t, &s->d2, &s->d2t, &s->d1, &s->d1t};
    for (bf16** a : acts) alloc(a, 2 * lt * kHid);  // row-major [mp][64] or transposed [64][ldt]
    // the hidden activations' transposes carry a row of ones (row 64) and zero rows up to 80:
    // the weight-gradient GEMMs then give each bias gradient as one more column
    bf16** tacts[] = {&s->h1t, &s->h2t, &s->h3t};
    for (bf16** a : tacts) alloc(a, 2 * lt * kTRows);
    alloc(&s->g4t, 2 * lt * kOut);
    alloc(&s->z, 4 * mp * kOut);
    alloc(&s->field, 4 * mp * kOut);
    alloc(&s->loss, 16);
    alloc(&s->status, 16);
    if (!ok) {
        mlp_destroy(s);
        return mlp_fail(WFPG_ERR_OOM, "mlp_create: device allocation failed");
    }
    if (params)
        ok = cudaMemcpyAsync(s->params, params, 4 * kParams, cudaMemcpyHostToDevice, st) == cudaSuccess;
    else
        ok = cudaMemsetAsync(s->params, 0, 4 * kParams, st) == cudaSuccess;
    for (bf16* t : {s->h1t, s->h2t, s->h3t}) {
        ok = ok && cudaMemsetAsync(t, 0, 2 * lt * kTRows, st) == cudaSuccess;
        if (ok) WFPG_LAUNCH(k_fill_bf16, div_up(lt, 256), 256, 0, st, t + (size_t)kHid * lt, (uint32_t)lt, 1.0f);
    }
    ok = ok && cudaMemsetAsync(s->m, 0, 4 * kParams, st) == cudaSuccess &&
         cudaMemsetAsync(s->v, 0, 4 * kParams, st) == cudaSuccess &&
         cudaMemsetAsync(s->status, 0, 16, st) == cudaSuccess;
    convert_weights(s, st);
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        mlp_destroy(s);
        return mlp_fail(WFPG_ERR_CUDA, "mlp_create: initialisation failed");
    }
    *out = s;
    return WFPG_OK;
}

int mlp_destroy(wfpg_mlp* s) {
    if (!s) return WFPG_OK;
    void* ptrs[] = {s->params, s->m, s->v, s->grad, s->part, s->w1, s->w2, s->w3, s->w4, s->w2t, s->w3t, s->w4t,
                    s->xt, s->h1, s->h1t, s->h2, s->h2t, s->h3, s->h3t, s->g4t, s->d3,
                    s->d3t, s->d2, s->d2t, s->d1, s->d1t, s->z, s->field, s->loss, s->status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete s;
    return WFPG_OK;
}

int mlp_get_params(const wfpg_mlp* s, float* params, void* stream) {
    if (!s || !params) return mlp_fail(WFPG_ERR_INVALID_ARG, "mlp_get_params: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(params, s->params, 4 * kParams, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return mlp_fail(WFPG_ERR_CUDA, "mlp_get_params: copy failed");
    return WFPG_OK;
}

int mlp_status(wfpg_mlp* s, uint32_t* flags, int clear, void* stream) {
    if (!s || !flags) return mlp_fail(WFPG_ERR_INVALID_ARG, "mlp_status: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(flags, s->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return mlp_fail(WFPG_ERR_CUDA, "mlp_status: copy failed");
    if (clear && cudaMemsetAsync(s->status, 0, 4, st) != cudaSuccess)
        return mlp_fail(WFPG_ERR_CUDA, "mlp_status: clear failed");
    return WFPG_OK;
}

int guide_learned_build_pdf(wfpg_mlp* s, const float* pos, const float* nrm, const uint32_t* origin_ray,
                            const uint32_t* n_bins_dev, uint32_t bin_cap, const wfpg_learned_params* p, float* pdf,
                            float* cdf_row, float* cdf_marg, void* stream) {
    if (!s || !p || !pos || !nrm) return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_build_pdf: null argument");
    if (bin_cap > s->max_batch)
        return mlp_fail(WFPG_ERR_CAPACITY, "guide_learned_build_pdf: bin_cap exceeds the MLP's max_batch");
    if (!(p->size > 0.0f) || !(p->eps >= 0.0f))
        return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_build_pdf: size must be > 0 and eps >= 0");
    if (bin_cap == 0) return WFPG_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hidden(s, pos, nrm, origin_ray, n_bins_dev, bin_cap, p, false, st);
    // the output layer fused with the softmax: field = softmax(logits) + eps, no logits stored
    alignas(64) CUtensorMap mh, mw;
    if (tensor_map(&mh, s->h3, kHid, (int)bin_cap, kHid, 128) && tensor_map(&mw, s->w4, kHid, kOut, kHid, 64)) {
        InferArgs ia{s->params + kOffB4, (int)bin_cap, p->eps, s->field, s->status};
        WFPG_LAUNCH(k_out_infer, div_up(bin_cap, 128), kOutThreads, kInferSmemBytes + 1024, st, mh, mw, ia);
    } else {
        g_gemm_failed = true;
    }
    if (wfpg::field_pdf_impl(s->field, 32, n_bins_dev, bin_cap, pdf, cdf_row, cdf_marg, st) != WFPG_OK ||
        cudaGetLastError() != cudaSuccess || gemm_failed())
        return mlp_fail(WFPG_ERR_CUDA, "guide_learned_build_pdf: launch failed");
    return WFPG_OK;
}

int guide_learned_logits(wfpg_mlp* s, const float* pos, const float* nrm, uint32_t n, const wfpg_learned_params* p,
                         float* logits, void* stream) {
    if (!s || !p || !pos || !nrm || !logits)
        return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_logits: null argument");
    if (n == 0 || n > s->max_batch)
        return mlp_fail(WFPG_ERR_CAPACITY, "guide_learned_logits: n must be in [1, max_batch]");
    if (!(p->size > 0.0f)) return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_logits: size must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hidden(s, pos, nrm, nullptr, nullptr, n, p, false, st);
    output_logits(s, (int)n, st, logits);
    if (cudaGetLastError() != cudaSuccess || gemm_failed())
        return mlp_fail(WFPG_ERR_CUDA, "guide_learned_logits: launch failed");
    return WFPG_OK;
}

int mlp_adam_step(wfpg_mlp* s, const float* grad, const wfpg_adam_params* opt, void* stream) {
    if (!s || !grad || !opt) return mlp_fail(WFPG_ERR_INVALID_ARG, "mlp_adam_step: null argument");
    if (!(opt->lr >= 0.0f) || !(opt->beta1 >= 0.0f && opt->beta1 < 1.0f) || !(opt->beta2 >= 0.0f && opt->beta2 < 1.0f) ||
        !(opt->eps >= 0.0f))
        return mlp_fail(WFPG_ERR_INVALID_ARG, "mlp_adam_step: need lr >= 0, beta1 and beta2 in [0, 1), eps >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    adam_update(s, grad, *opt, st);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(WFPG_ERR_CUDA, "mlp_adam_step: launch failed");
    return WFPG_OK;
}

int guide_learned_train_step(wfpg_mlp* s, const float* pos, const float* nrm, uint32_t n, const float* target,
                             const wfpg_learned_params* p, const wfpg_adam_params* opt, float* loss_out,
                             float* grad_out, void* stream) {
    if (!s || !p || !opt) return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_train_step: null argument");
    if (!pos || !nrm || !target) return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_train_step: null array");
    if (reinterpret_cast<uintptr_t>(target) % 32 != 0)
        return mlp_fail(WFPG_ERR_INVALID_ARG, "guide_learned_train_step: target must be 32-byte aligned");
    if (n == 0 || n > s->max_batch)
        return mlp_fail(WFPG_ERR_CAPACITY, "guide_learned_train_step: n must be in [1, max_batch]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int lt = (int)s->ldt, N = (int)n;
    bool ok = cudaMemsetAsync(s->grad, 0, 4 * kParams, st) == cudaSuccess &&
              cudaMemsetAsync(s->loss, 0, 4, st) == cudaSuccess;
    hidden(s, pos, nrm, nullptr, nullptr, n, p, true, st);
    // output layer, fused: logits, softmax, KL, G4^T, db4 and dA3 = (G4 W4) o [H3 > 0] per 128-row tile
    {
        static std::atomic<uint64_t> raised{0};
        int dev = 0;
        cudaGetDevice(&dev);
        const uint64_t bit = 1ull << (dev & 63);
        if (!(raised.load(std::memory_order_relaxed) & bit)) {
            cudaFuncSetAttribute(k_out_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kOutSmemBytes + 1024);
            raised.fetch_or(bit, std::memory_order_relaxed);
        }
        OutTrainArgs oa;
        oa.h3 = s->h3;
        oa.w4 = s->w4;
        oa.w4t = s->w4t;
        oa.b4 = s->params + kOffB4;
        oa.target = target;
        oa.n = N;
        oa.inv_n = 1.0f / (float)n;
        oa.g4t = s->g4t;
        oa.ldg = lt;
        oa.d3 = s->d3;
        oa.d3t = s->d3t;
        oa.loss = s->loss;
        oa.status = s->status;
        // TMA maps: H3 tiles of 128 rows, W4 row blocks and W4^T column blocks of 64 x 64
        alignas(64) CUtensorMap mh, mw, mwt;
        if (tensor_map(&mh, s->h3, kHid, N, kHid, 128) && tensor_map(&mw, s->w4, kHid, kOut, kHid, 64) &&
            tensor_map(&mwt, s->w4t, kOut, kHid, kOut, 64))
            WFPG_LAUNCH(k_out_train, div_up(n, 128), kOutThreads, kOutSmemBytes + 1024, st, mh, mw, mwt, oa);
        else
            g_gemm_failed = true;
    }
    // [dW4 | db4] = G4^T [H3 | 1] (split-K over the batch; H3^T carries a row of ones)
    GemmArgs g = gargs(s->g4t, lt, s->h3t, lt, kOut, kTRows, N, s->status);
    weight_grad_wb(s, g, s->grad + kOffW4, kHid, kHid, s->grad + kOffB4, kHid, st);
    // hidden layers
    struct Layer {
        bf16 *dA, *dAt, *Hprev_t, *Hprev, *Wt, *dAprev, *dAprev_t;
        size_t offW, offB;
        int nin;
    } L[3] = {{s->d3, s->d3t, s->h2t, s->h2, s->w3t, s->d2, s->d2t, kOffW3, kOffB3, kHid},
              {s->d2, s->d2t, s->h1t, s->h1, s->w2t, s->d1, s->d1t, kOffW2, kOffB2, kHid},
              {s->d1, s->d1t, s->xt, nullptr, nullptr, nullptr, nullptr, kOffW1, kOffB1, kIn}};
    for (int l = 0; l < 3; ++l) {
        // [dW | db] = dA^T [H_prev | 1]: the bias gradient is the column of the ones row
        // (row 64 of the hidden transposes, padding row 78 of X^T)
        g = gargs(L[l].dAt, lt, L[l].Hprev_t, lt, kHid, kTRows, N, s->status);
        const int wcols = L[l].nin == kIn ? kFeatIn : kHid, ones = L[l].nin == kIn ? kFeatIn : kHid;
        weight_grad_wb(s, g, s->grad + L[l].offW, L[l].nin, wcols, s->grad + L[l].offB, ones, st);
        if (L[l].Wt) {
            g = gargs(L[l].dA, kHid, L[l].Wt, kHid, N, kHid, kHid, s->status);
            g.O = L[l].dAprev;
            g.ldo = kHid;
            g.OT = L[l].dAprev_t;
            g.ldot = lt;
            g.act = L[l].Hprev;
            g.ldact = kHid;
            gemm<64, kEpiReluGrad>(g, 1, st);
        }
    }
    if (grad_out) ok = ok && cudaMemcpyAsync(grad_out, s->grad, 4 * kParams, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    if (loss_out) ok = ok && cudaMemcpyAsync(loss_out, s->loss, 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    if (opt->update) adam_update(s, s->grad, *opt, st);
    if (!ok || cudaGetLastError() != cudaSuccess || gemm_failed())
        return mlp_fail(WFPG_ERR_CUDA, "guide_learned_train_step: launch failed");
    return WFPG_OK;
}

}  // extern "C"
