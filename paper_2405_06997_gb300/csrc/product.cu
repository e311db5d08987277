// Product path guiding (Sec. 3.6): the bin's field at 8 x 8 blocks times the
// ray's BSDF at the same resolution, sampled in two stages -- a block from the
// product, then a cell and a point in it from the full-resolution field inside
// the block (the paper does this with a warp per ray; here one thread takes a
// ray, the 64 block directions are shared through shared memory, and every
// sum runs in a fixed sequential order).
//
//   S_B    = sum of the cell densities of block B (b x b cells, b = N / 8), row-major;
//   beta_B = max(0, n . w_B) + 2^-10, w_B the octahedral image of the block centre;
//   Z      = running sum of beta_B S_B over the 64 blocks (row-major);
//   p(w)   = beta_B pdf_c N^2 / (4 pi Z).
#include "common.cuh"

namespace wfpg {

constexpr float kProductKappa = 0x1p-10f;
constexpr float kProductOneMinus = 0x1.fffffep-1f;

__device__ __forceinline__ float unit_clamp(float x) {
    if (!(x >= 0.0f)) return 0.0f;
    return x >= 1.0f ? kProductOneMinus : x;
}

// S[bin][B]: one thread per (bin, block), the block's cells summed row by row
__global__ void __launch_bounds__(64) k_product_sums(const float* __restrict__ pdf, int N,
                                                    const uint32_t* __restrict__ n_bins_dev, uint32_t bin_cap,
                                                    float* __restrict__ S) {
    const uint32_t bin = blockIdx.x;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    if (bin >= nb) return;
    const int B = threadIdx.x, bi = B & 7, bj = B >> 3, b = N >> 3;
    const float* f = pdf + (size_t)bin * N * N;
    float s = 0.0f;
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) s = __fadd_rn(s, f[(bj * b + r) * N + bi * b + c]);
    S[(size_t)bin * 64 + B] = s;
}

__device__ __forceinline__ void load_block_dirs(float* s_dir) {
    for (int B = threadIdx.x; B < 64; B += blockDim.x) {
        const float u = __fsub_rn(__fmul_rn(__fadd_rn((float)(B & 7), 0.5f), 0.25f), 1.0f);
        const float v = __fsub_rn(__fmul_rn(__fadd_rn((float)(B >> 3), 0.5f), 0.25f), 1.0f);
        const float3 d = octa_to_dir(u, v);
        s_dir[3 * B] = d.x;
        s_dir[3 * B + 1] = d.y;
        s_dir[3 * B + 2] = d.z;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_weight(const float* s_dir, int B, float nx, float ny, float nz) {
    const float dot = __fadd_rn(__fadd_rn(__fmul_rn(nx, s_dir[3 * B]), __fmul_rn(ny, s_dir[3 * B + 1])),
                                __fmul_rn(nz, s_dir[3 * B + 2]));
    return __fadd_rn(fmaxf(dot, 0.0f), kProductKappa);
}

__device__ __forceinline__ float product_density(float beta, float pdf_c, int N, float Z) {
    return __fdiv_rn(__fmul_rn(__fmul_rn(beta, pdf_c), (float)(N * N)), __fmul_rn(Z, 12.566370614359172f));
}

// Z for a normal; with Bsel, also the block holding the running-sum target t
// (first B with C_B > t, else 63) and its bounds C_{B-1}, C_B
__device__ __forceinline__ float product_norm(const float* s_dir, const float* Sb, float nx, float ny, float nz,
                                              float u0, int* Bsel, float* lo, float* hi) {
    float acc = 0.0f;
    for (int B = 0; B < 64; ++B) acc = __fadd_rn(acc, __fmul_rn(block_weight(s_dir, B, nx, ny, nz), Sb[B]));
    if (Bsel) {
        const float t = __fmul_rn(u0, acc);
        float run = 0.0f, prev = 0.0f;
        int sel = 63;
        for (int B = 0; B < 64; ++B) {
            prev = run;
            run = __fadd_rn(run, __fmul_rn(block_weight(s_dir, B, nx, ny, nz), Sb[B]));
            if (run > t) {
                sel = B;
                break;
            }
        }
        *Bsel = sel;
        *lo = prev;
        *hi = run;
    }
    return acc;
}

// one ray: product sample if u2 < alpha, else cosine; mixture density
__global__ void __launch_bounds__(256) k_product_sample(const float* __restrict__ pdf, const float* __restrict__ S,
                                                        int N, uint32_t bin_cap, const uint32_t* __restrict__ n_bins_dev,
                                                        const uint32_t* __restrict__ bin_of_ray,
                                                        const float* __restrict__ nrm, const float* __restrict__ u,
                                                        uint32_t n_cap, const uint32_t* __restrict__ n_dev,
                                                        float alpha, float* __restrict__ dir,
                                                        float* __restrict__ pdf_out, uint32_t* __restrict__ cell) {
    __shared__ float s_dir[192];
    load_block_dirs(s_dir);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = n_dev ? min(*n_dev, n_cap) : n_cap;
    if (i >= n) return;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const uint32_t bin = bin_of_ray[i];
    const float u0 = u[3 * (size_t)i], u1 = u[3 * (size_t)i + 1], u2 = u[3 * (size_t)i + 2];
    const float nx = nrm[3 * (size_t)i], ny = nrm[3 * (size_t)i + 1], nz = nrm[3 * (size_t)i + 2];
    float3 d;
    float pp = 0.0f, a = alpha;
    uint32_t cl = kNone;
    if (bin >= nb) {
        a = 0.0f;
        d = cosine_dir(nx, ny, nz, u0, u1);
    } else {
        const float* f = pdf + (size_t)bin * N * N;
        const float* Sb = S + (size_t)bin * 64;
        if (u2 < alpha) {
            int B;
            float lo, hi;
            const float Z = product_norm(s_dir, Sb, nx, ny, nz, u0, &B, &lo, &hi);
            const float t = __fmul_rn(u0, Z);
            const float u0p = unit_clamp(__fdiv_rn(__fsub_rn(t, lo), __fsub_rn(hi, lo)));
            const int b = N >> 3, i0 = (B & 7) * b, j0 = (B >> 3) * b;
            // rows of the block: running sum of the row sums (b <= 16)
            float CR[16];
            float acc = 0.0f;
            for (int k = 0; k < b; ++k) {
                float s = 0.0f;
                for (int c = 0; c < b; ++c) s = __fadd_rn(s, f[(j0 + k) * N + i0 + c]);
                acc = __fadd_rn(acc, s);
                CR[k] = acc;
            }
            const float t0 = __fmul_rn(u0p, CR[b - 1]);
            int r = b - 1;
            for (int k = 0; k < b; ++k)
                if (CR[k] > t0) {
                    r = k;
                    break;
                }
            const float rlo = r > 0 ? CR[r - 1] : 0.0f, rhi = CR[r];
            const float beta_r = unit_clamp(__fdiv_rn(__fsub_rn(t0, rlo), __fsub_rn(rhi, rlo)));
            // cells of the chosen row: running sum, first above u1 * row total
            float rowtot = 0.0f;
            for (int c = 0; c < b; ++c) rowtot = __fadd_rn(rowtot, f[(j0 + r) * N + i0 + c]);
            const float t1 = __fmul_rn(u1, rowtot);
            int c = b - 1;
            float clo = 0.0f, chi = 0.0f, run = 0.0f;
            for (int k = 0; k < b; ++k) {
                const float prev = run;
                run = __fadd_rn(run, f[(j0 + r) * N + i0 + k]);
                clo = prev;
                chi = run;
                if (run > t1) {
                    c = k;
                    break;
                }
            }
            const float al = unit_clamp(__fdiv_rn(__fsub_rn(t1, clo), __fsub_rn(chi, clo)));
            const float tn = __fdiv_rn(2.0f, (float)N);
            d = octa_to_dir(__fsub_rn(__fmul_rn(__fadd_rn((float)(i0 + c), al), tn), 1.0f),
                            __fsub_rn(__fmul_rn(__fadd_rn((float)(j0 + r), beta_r), tn), 1.0f));
            cl = (uint32_t)((j0 + r) * N + i0 + c);
            pp = product_density(block_weight(s_dir, B, nx, ny, nz), f[cl], N, Z);
        } else {
            d = cosine_dir(nx, ny, nz, u0, u1);
            const float Z = product_norm(s_dir, Sb, nx, ny, nz, 0.0f, nullptr, nullptr, nullptr);
            const int c = octa_cell(d, N);
            const int b = N >> 3;
            const int B = ((c / N) / b) * 8 + (c % N) / b;
            pp = product_density(block_weight(s_dir, B, nx, ny, nz), f[c], N, Z);
        }
    }
    const float cs = fmaxf(0.0f, nx * d.x + ny * d.y + nz * d.z);
    dir[3 * (size_t)i] = d.x;
    dir[3 * (size_t)i + 1] = d.y;
    dir[3 * (size_t)i + 2] = d.z;
    pdf_out[i] = a * pp + (1.0f - a) * cs * 0.31830988618379067f;
    if (cell) cell[i] = cl;
}

// mixture density of given directions: alpha * product + (1 - alpha) * cos+ / pi
__global__ void __launch_bounds__(256) k_product_eval(const float* __restrict__ pdf, const float* __restrict__ S,
                                                      int N, uint32_t bin_cap, const uint32_t* __restrict__ n_bins_dev,
                                                      const uint32_t* __restrict__ bin, const float* __restrict__ nrm,
                                                      const float* __restrict__ dir, uint32_t n_cap,
                                                      const uint32_t* __restrict__ n_dev, float alpha,
                                                      float* __restrict__ out) {
    __shared__ float s_dir[192];
    load_block_dirs(s_dir);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = n_dev ? min(*n_dev, n_cap) : n_cap;
    if (i >= n) return;
    const uint32_t nb = n_bins_dev ? min(*n_bins_dev, bin_cap) : bin_cap;
    const float nx = nrm[3 * (size_t)i], ny = nrm[3 * (size_t)i + 1], nz = nrm[3 * (size_t)i + 2];
    const float dx = dir[3 * (size_t)i], dy = dir[3 * (size_t)i + 1], dz = dir[3 * (size_t)i + 2];
    const float cs = fmaxf(0.0f, nx * dx + ny * dy + nz * dz);
    const uint32_t b_ = bin[i];
    float a = alpha, pp = 0.0f;
    if (b_ >= nb) {
        a = 0.0f;
    } else {
        const float Z = product_norm(s_dir, S + (size_t)b_ * 64, nx, ny, nz, 0.0f, nullptr, nullptr, nullptr);
        const int c = octa_cell(make_float3(dx, dy, dz), N);
        const int b = N >> 3;
        const int B = ((c / N) / b) * 8 + (c % N) / b;
        pp = product_density(block_weight(s_dir, B, nx, ny, nz), pdf[(size_t)b_ * N * N + c], N, Z);
    }
    out[i] = a * pp + (1.0f - a) * cs * 0.31830988618379067f;
}

int product_sums_impl(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, float* S,
                      cudaStream_t st) {
    if (bin_cap == 0) return WFPG_OK;
    WFPG_LAUNCH(k_product_sums, bin_cap, 64, 0, st, pdf, N, n_bins_dev, bin_cap, S);
    return launch_status();
}

int product_sample_impl(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                        const uint32_t* bin_of_ray, const float* nrm, const float* u, uint32_t n,
                        const uint32_t* n_dev, float alpha, float* dir, float* pdf_out, uint32_t* cell,
                        cudaStream_t st) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_product_sample, div_up(n, 256), 256, 0, st, pdf, S, N, bin_cap, n_bins_dev, bin_of_ray, nrm, u, n,
                n_dev, alpha, dir, pdf_out, cell);
    return launch_status();
}

int product_eval_impl(const float* pdf, const float* S, int N, uint32_t bin_cap, const uint32_t* n_bins_dev,
                      const uint32_t* bin, const float* nrm, const float* dir, uint32_t n, float alpha, float* out,
                      cudaStream_t st, const uint32_t* n_dev) {
    if (n == 0) return WFPG_OK;
    WFPG_LAUNCH(k_product_eval, div_up(n, 256), 256, 0, st, pdf, S, N, bin_cap, n_bins_dev, bin, nrm, dir, n, n_dev,
                alpha, out);
    return launch_status();
}

}  // namespace wfpg
