// CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// Product path guiding (Sec. 3.6): the bin's radiance field is down-sampled to
// an 8 x 8 grid of blocks, multiplied block by block with the ray's BSDF
// field at that resolution, and sampled in two stages -- a block from the
// product, then a cell (and a point in it) from the full-resolution field
// inside the block.  Written from the section's description, in this order:
//
//   S_B    = sum of the field's cell densities pdf_c over the b x b cells of
//            block B (b = N / 8), row-major, left to right;
//   beta_B = max(0, n . w_B) + 2^-10, w_B the octahedral image of the block's
//            centre (the Lambertian BSDF at the block; the floor keeps the
//            product positive wherever the field is);
//   C_B    = running sum of beta_B S_B over B = 0..63 (row-major blocks),
//            Z = C_63;
//   block  = first B with C_B > u0 Z; its remainder u0' continues below;
//   inside the block: row sums R_r, their running sum, row = first > u0' R,
//            then the running sum of that row's cells, column = first > u1 R_r,
//            with the in-cell offsets by linear inversion (as in Alg. 3's
//            sampler);
//   density p(w) = beta_B pdf_c N^2 / (4 pi Z)  (sums to 1 over the sphere).
//
// Every step is binary32 with one rounding per written operation.
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "oracle_internal.h"

namespace orc {

static constexpr float kFourPi = 12.566370614359172f;
static constexpr float kKappa = 0x1p-10f;  // 2^-10

static float clamp_unit(float x) {
    if (!(x >= 0.0f)) return 0.0f;
    return x >= 1.0f ? 0x1.fffffep-1f : x;
}

// centre direction of block (bi, bj) of the 8 x 8 grid
static void block_dir(int bi, int bj, float d[3]) {
    const float u = ((float)bi + 0.5f) * 0.25f - 1.0f;
    const float v = ((float)bj + 0.5f) * 0.25f - 1.0f;
    octa_decode(u, v, d);
}

void product_block_sums(const float* pdf, int N, float S[64]) {
    const int b = N / 8;
    for (int bj = 0; bj < 8; ++bj)
        for (int bi = 0; bi < 8; ++bi) {
            float s = 0.0f;
            for (int r = 0; r < b; ++r)
                for (int c = 0; c < b; ++c) s = s + pdf[(bj * b + r) * N + bi * b + c];
            S[bj * 8 + bi] = s;
        }
}

float product_block_weight(const float n[3], int B) {
    float d[3];
    block_dir(B % 8, B / 8, d);
    const float dot = (n[0] * d[0] + n[1] * d[1]) + n[2] * d[2];
    return std::max(dot, 0.0f) + kKappa;
}

static float product_norm(const float* S, const float n[3], float C[64]) {
    float acc = 0.0f;
    for (int B = 0; B < 64; ++B) {
        acc = acc + product_block_weight(n, B) * S[B];
        C[B] = acc;
    }
    return acc;
}

static float product_density(float beta, float pdf_c, int N, float Z) {
    const float num = (beta * pdf_c) * (float)(N * N);
    return num / (Z * kFourPi);
}

void product_sample_one(const float* pdf, const float* S, int N, const float n[3], float u0, float u1,
                        float dir[3], float* p, uint32_t* cell) {
    float C[64];
    const float Z = product_norm(S, n, C);
    const float t = u0 * Z;
    int B = 63;
    for (int k = 0; k < 64; ++k)
        if (C[k] > t) { B = k; break; }
    const float lo = B > 0 ? C[B - 1] : 0.0f;
    const float u0p = clamp_unit((t - lo) / (C[B] - lo));
    const int b = N / 8, i0 = (B % 8) * b, j0 = (B / 8) * b;
    float CR[16] = {};
    float acc = 0.0f;
    for (int r = 0; r < b; ++r) {
        float s = 0.0f;
        for (int c = 0; c < b; ++c) s = s + pdf[(j0 + r) * N + i0 + c];
        acc = acc + s;
        CR[r] = acc;
    }
    const float t0 = u0p * CR[b - 1];
    int r = b - 1;
    for (int k = 0; k < b; ++k)
        if (CR[k] > t0) { r = k; break; }
    const float rlo = r > 0 ? CR[r - 1] : 0.0f;
    const float beta_r = clamp_unit((t0 - rlo) / (CR[r] - rlo));
    float CC[16] = {};
    acc = 0.0f;
    for (int c = 0; c < b; ++c) {
        acc = acc + pdf[(j0 + r) * N + i0 + c];
        CC[c] = acc;
    }
    const float t1 = u1 * CC[b - 1];
    int c = b - 1;
    for (int k = 0; k < b; ++k)
        if (CC[k] > t1) { c = k; break; }
    const float clo = c > 0 ? CC[c - 1] : 0.0f;
    const float alpha = clamp_unit((t1 - clo) / (CC[c] - clo));
    const float tn = 2.0f / (float)N;
    const float u = ((float)(i0 + c) + alpha) * tn - 1.0f;
    const float v = ((float)(j0 + r) + beta_r) * tn - 1.0f;
    octa_decode(u, v, dir);
    const uint32_t cl = (uint32_t)((j0 + r) * N + i0 + c);
    *cell = cl;
    *p = product_density(product_block_weight(n, B), pdf[cl], N, Z);
}

float product_eval_one(const float* pdf, const float* S, int N, const float n[3], const float d[3]) {
    float C[64];
    const float Z = product_norm(S, n, C);
    float u, v;
    octa_encode(d, &u, &v);
    const float hn = (float)N * 0.5f;
    const float a = (u + 1.0f) * hn, bb = (v + 1.0f) * hn;
    const int i = std::min((a >= 0.0f) ? (int)a : 0, N - 1);
    const int j = std::min((bb >= 0.0f) ? (int)bb : 0, N - 1);
    const int b = N / 8;
    const int B = (j / b) * 8 + i / b;
    return product_density(product_block_weight(n, B), pdf[j * N + i], N, Z);
}

}  // namespace orc

extern "C" {

void orc_product_block_sums(const float* pdf, int N, size_t bins, float* S) {
    const size_t NN = (size_t)N * N;
    for (size_t k = 0; k < bins; ++k) orc::product_block_sums(pdf + k * NN, N, S + 64 * k);
}

void orc_product_sample(const float* pdf, const float* S, int N, const uint32_t* bin, const float* nrm,
                        const float* u, size_t n, float* dir, float* p, uint32_t* cell) {
    const size_t NN = (size_t)N * N;
    for (size_t i = 0; i < n; ++i)
        orc::product_sample_one(pdf + bin[i] * NN, S + 64 * (size_t)bin[i], N, nrm + 3 * i, u[2 * i],
                                u[2 * i + 1], dir + 3 * i, p + i, cell + i);
}

void orc_product_eval(const float* pdf, const float* S, int N, const uint32_t* bin, const float* nrm,
                      const float* dir, size_t n, float* out) {
    const size_t NN = (size_t)N * N;
    for (size_t i = 0; i < n; ++i)
        out[i] = orc::product_eval_one(pdf + bin[i] * NN, S + 64 * (size_t)bin[i], N, nrm + 3 * i, dir + 3 * i);
}

float orc_product_block_weight(const float* n, int B) { return orc::product_block_weight(n, B); }

}  // extern "C"
