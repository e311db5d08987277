// CPU ORACLE -- TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
//
// GuideRays (Alg. 3): the per-bin radiance field, its PDF and CDF (Sec. 3.5
// "Path Guiding", Sec. 3 "Implementation": jitter, Gaussian blur, epsilon
// floor), inverse-CDF sampling and PDF evaluation.
#include <algorithm>
#include <cmath>
#include <vector>

#include "oracle_internal.h"

namespace orc {

static constexpr float FOUR_PI = 12.566370614359172f;
static constexpr float ONE_MINUS = 0x1.fffffep-1f;

// Field of one bin: cell (i, j) -- column i along u, row j along v -- covers
// u in [2i/N - 1, 2(i+1)/N - 1] (same for v, j).  Its query direction is the
// octahedral image of the cell centre, or of a jittered point in the cell
// (xi from the counter generator, stream (frame, bin), counters 2c and 2c+1
// for cell c = j*N + i).  The field starts at eps everywhere (the paper's
// epsilon = 1e-2) and the cone-traced radiance is added.
void build_field(const Svo& s, const float o[3], uint32_t bin, int N, float eps, int jitter,
                 float t_skip, int cos_weight, uint64_t seed, uint32_t frame, float* f,
                 uint64_t* steps, uint64_t* blocks) {
    const float omega = FOUR_PI / (float)(N * N);
    const float tn = 2.0f / (float)N;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            uint32_t c = (uint32_t)(j * N + i);
            float x0 = 0.5f, x1 = 0.5f;
            if (jitter) {
                x0 = rng_unit(purpose_seed(seed, PURPOSE_JITTER), bin_stream(frame, bin), 2ull * c);
                x1 = rng_unit(purpose_seed(seed, PURPOSE_JITTER), bin_stream(frame, bin), 2ull * c + 1);
            }
            float u = ((float)i + x0) * tn - 1.0f;
            float v = ((float)j + x1) * tn - 1.0f;
            float d[3];
            octa_decode(u, v, d);
            TraceResult r = trace_cell(s, o, d, t_skip, omega, cos_weight, blocks != nullptr);
            if (steps) *steps += r.steps;
            if (blocks) *blocks += r.blocks;
            f[c] = eps + r.value;
        }
}

// Blur (the paper's "Gaussian blur" of the field).  Reading: separable 3-tap
// binomial [1 2 1]/4, first along v (rows) then along u (columns).  Off the
// square's edge the octahedral map continues mirrored: row -1 of column i is
// row 0 of column N-1-i, row N is row N-1 of column N-1-i, and likewise for
// columns.
void blur_field(float* f, int N) {
    std::vector<float> t(N * N);
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            float up = (j > 0) ? f[(j - 1) * N + i] : f[0 * N + (N - 1 - i)];
            float dn = (j < N - 1) ? f[(j + 1) * N + i] : f[(N - 1) * N + (N - 1 - i)];
            float b = f[j * N + i];
            t[j * N + i] = ((up + dn) + (b + b)) * 0.25f;
        }
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            float lf = (i > 0) ? t[j * N + i - 1] : t[(N - 1 - j) * N + 0];
            float rt = (i < N - 1) ? t[j * N + i + 1] : t[(N - 1 - j) * N + (N - 1)];
            float b = t[j * N + i];
            f[j * N + i] = ((lf + rt) + (b + b)) * 0.25f;
        }
}

// Inclusive prefix sum in the order the paper's warp scan produces it
// (Sec. 3.5): the sequence is cut into chunks of 32 (one warp each); inside a
// chunk, rounds k = 1, 2, 4, 8, 16 replace x[i] by x[i] + x[i-k] for every
// i >= k at once; each later chunk then adds the running total on its left.
void warp_order_scan(float* x, int n) {
    const int W = n < 32 ? n : 32;
    float carry = 0.0f;
    std::vector<float> nx(W);
    for (int c0 = 0; c0 < n; c0 += W) {
        float* y = x + c0;
        for (int k = 1; k < W; k *= 2) {
            for (int i = 0; i < W; ++i) nx[i] = (i >= k) ? y[i] + y[i - k] : y[i];
            for (int i = 0; i < W; ++i) y[i] = nx[i];
        }
        if (c0 > 0)
            for (int i = 0; i < W; ++i) y[i] = carry + y[i];
        carry = y[W - 1];
    }
}

// A CDF is the warp-order scan followed by a running maximum.  The running
// maximum is exact and changes nothing unless rounding in the tree-shaped scan
// made an entry smaller than the one before it; it keeps every CDF
// non-decreasing, as a CDF is by definition, so "the first entry greater than
// t" can be found by bisection.
static void cdf_scan(float* x, int n) {
    warp_order_scan(x, n);
    for (int i = 1; i < n; ++i) x[i] = std::max(x[i], x[i - 1]);
}

// GeneratePDF-CDF (Alg. 3): the field as a piecewise-constant density on the
// sphere.  Row CDFs (inclusive), then the marginal CDF over row totals; the
// density of cell c is f_c / T * N^2 / (4 pi) (each cell spans 4 pi / N^2 sr).
void pdf_cdf(const float* f, int N, float* pdf, float* cdf_row, float* cdf_marg) {
    std::vector<float> rt(N);
    for (int j = 0; j < N; ++j) {
        for (int i = 0; i < N; ++i) cdf_row[j * N + i] = f[j * N + i];
        cdf_scan(cdf_row + j * N, N);
        rt[j] = cdf_row[j * N + N - 1];
    }
    for (int j = 0; j < N; ++j) cdf_marg[j] = rt[j];
    cdf_scan(cdf_marg, N);
    float T = cdf_marg[N - 1];
    float nn = (float)(N * N);
    float den = T * FOUR_PI;
    for (int c = 0; c < N * N; ++c) pdf[c] = (f[c] * nn) / den;
}

static float clamp01(float x) {
    if (!(x >= 0.0f)) return 0.0f;
    return x >= 1.0f ? ONE_MINUS : x;
}

// Inverse-CDF sampling of the piecewise-constant 2D density (Alg. 3 "MIS",
// the guided branch): u0 picks the row (first marginal entry > u0 * T),
// u1 the column within it (first row-CDF entry > u1 * T_row), both clamped to
// N - 1; the position inside the cell is the linear inverse of the CDF
// across it.  Returns the direction, the cell's density and the cell index.
void sample_one(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, float u0,
                float u1, float dir[3], float* p, uint32_t* cell) {
    float t0 = u0 * cdf_marg[N - 1];
    int r = N - 1;
    for (int j = 0; j < N; ++j)
        if (cdf_marg[j] > t0) { r = j; break; }
    const float* C = cdf_row + r * N;
    float t1 = u1 * C[N - 1];
    int c = N - 1;
    for (int i = 0; i < N; ++i)
        if (C[i] > t1) { c = i; break; }
    float mlo = r > 0 ? cdf_marg[r - 1] : 0.0f, mhi = cdf_marg[r];
    float clo = c > 0 ? C[c - 1] : 0.0f, chi = C[c];
    float beta = clamp01((t0 - mlo) / (mhi - mlo));
    float alpha = clamp01((t1 - clo) / (chi - clo));
    const float tn = 2.0f / (float)N;
    float u = ((float)c + alpha) * tn - 1.0f;
    float v = ((float)r + beta) * tn - 1.0f;
    octa_decode(u, v, dir);
    *cell = (uint32_t)(r * N + c);
    *p = pdf[r * N + c];
}

// PDF of an arbitrary direction (needed by MIS): its cell under the
// octahedral map, i = floor((u + 1) N / 2) clamped to [0, N-1], same for j.
float eval_one(const float* pdf, int N, const float d[3]) {
    float u, v;
    octa_encode(d, &u, &v);
    const float hn = (float)N * 0.5f;
    float a = (u + 1.0f) * hn, b = (v + 1.0f) * hn;
    int i = (a >= 0.0f) ? (int)a : 0;
    int j = (b >= 0.0f) ? (int)b : 0;
    i = std::min(i, N - 1);
    j = std::min(j, N - 1);
    return pdf[j * N + i];
}

}  // namespace orc
