// Shared device helpers of the wfpg CUDA library (sm_103a).
//
// Every floating-point step whose result decides an integer downstream (a
// voxel, the leaf a cone ray reaches, the cone level, a side, a sampled cell)
// is written with explicit round-to-nearest intrinsics (__fadd_rn, __fmul_rn,
// __fdiv_rn, __fsqrt_rn, ...), which the compiler never fuses or reorders, so
// that the result is one fixed IEEE binary32 sequence.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wfpg.h"

namespace wfpg {

constexpr uint32_t kNone = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// counter-based random numbers: SplitMix64's output function (Steele, Lea &
// Flood 2014) over key = mix(seed ^ stream * gamma), value = mix(key +
// (counter + 1) * gamma); the top 24 bits form a uniform on [0, 1).
__host__ __device__ __forceinline__ uint64_t splitmix_finalize(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;
__host__ __device__ __forceinline__ uint64_t counter_rng(uint64_t seed, uint64_t stream,
                                                         uint64_t counter) {
    const uint64_t key = splitmix_finalize(seed ^ (stream * kGamma));
    return splitmix_finalize(key + (counter + 1) * kGamma);
}
__device__ __forceinline__ uint32_t uniform24(uint64_t seed, uint64_t stream, uint64_t counter) {
    return (uint32_t)(counter_rng(seed, stream, counter) >> 40);
}
__device__ __forceinline__ float uniform01(uint64_t seed, uint64_t stream, uint64_t counter) {
    return __fmul_rn(__uint2float_rn(uniform24(seed, stream, counter)), 0x1p-24f);
}
// stream purposes folded into the seed
constexpr uint64_t kOriginPurpose = 0, kJitterPurpose = 1;
__host__ __device__ __forceinline__ uint64_t purpose(uint64_t seed, uint64_t p) { return seed * 4 + p; }
__host__ __device__ __forceinline__ uint64_t bin_stream(uint32_t frame, uint32_t bin) {
    return ((uint64_t)frame << 32) | bin;
}

// ---------------------------------------------------------------------------
// Morton keys: x bits at 3i, y at 3i+1, z at 3i+2 (21 bits per axis)
__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}
__host__ __device__ __forceinline__ uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ULL;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ULL;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00fULL;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffULL;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffULL;
    x = (x ^ (x >> 32)) & 0x1fffffULL;
    return (uint32_t)x;
}

// world coordinate -> leaf index: floor((x - lo) * scale) clamped, NaN -> 0
__device__ __forceinline__ int grid_index(float x, float lo, float scale, int D) {
    const float g = __fmul_rn(__fsub_rn(x, lo), scale);
    if (!(g >= 0.0f)) return 0;
    const int res = 1 << D;
    if (g >= (float)res) return res - 1;
    return (int)g;
}

// deepest level of the SVO's top index (a dense grid per level 0 .. this)
constexpr int kTopLevelMax = 6;
constexpr uint32_t kTopNodeMask = (1u << 28) - 1u;
// deepest SVO for which every level below the top index has an occupancy bitmap (8^l bits per
// level l: 1.2 GB in all at depth 11)
constexpr int kOccMaxDepth = 11;
// word offset of level l's bitmap when levels g + 1 .. l - 1 precede it (8^j bits each, j > 6)
__host__ __device__ __forceinline__ uint64_t occ_offset(int g, int l) {
    uint64_t o = 0;
    for (int j = g + 1; j < l; ++j) o += (1ull << (3 * j)) >> 5;
    return o;
}

// node record used by every tree walk: first child's global id and child mask
struct Node {
    uint32_t first_child;
    uint32_t mask;
};

// child slot of leaf cell c below a node at level l (D levels)
__device__ __forceinline__ int child_slot(const int c[3], int l, int D) {
    const int sh = D - 1 - l;
    return ((c[0] >> sh) & 1) | (((c[1] >> sh) & 1) << 1) | (((c[2] >> sh) & 1) << 2);
}
__device__ __forceinline__ uint32_t child_id(Node n, int k) {
    return n.first_child + __popc(n.mask & ((1u << k) - 1u));
}

// deepest existing node holding leaf cell c (Alg. 2 DescendLeaf); *level out
__device__ __forceinline__ uint32_t descend(const Node* __restrict__ nodes, const int c[3], int D,
                                            int* level) {
    uint32_t node = 0;
    int l = 0;
    while (l < D) {
        const Node n = nodes[node];
        const int k = child_slot(c, l, D);
        if (!((n.mask >> k) & 1u)) break;
        node = child_id(n, k);
        ++l;
    }
    *level = l;
    return node;
}

// ---------------------------------------------------------------------------
// own sine / cosine / arctangent from their Taylor series (coefficients are
// the binary32 roundings of 1/n! and 1/n), Horner in x^2, one rounding per op
__device__ __forceinline__ float taylor_sin(float x) {  // |x| <= pi/4
    const float x2 = __fmul_rn(x, x);
    float p = -0x1.ae6456p-26f;
    p = __fadd_rn(__fmul_rn(p, x2), 0x1.71de3ap-19f);
    p = __fadd_rn(__fmul_rn(p, x2), -0x1.a01a02p-13f);
    p = __fadd_rn(__fmul_rn(p, x2), 0x1.111112p-7f);
    p = __fadd_rn(__fmul_rn(p, x2), -0x1.555556p-3f);
    p = __fmul_rn(p, x2);
    return __fadd_rn(x, __fmul_rn(x, p));
}
__device__ __forceinline__ float taylor_cos(float x) {  // |x| <= pi/4
    const float x2 = __fmul_rn(x, x);
    float p = -0x1.27e4fcp-22f;
    p = __fadd_rn(__fmul_rn(p, x2), 0x1.a01a02p-16f);
    p = __fadd_rn(__fmul_rn(p, x2), -0x1.6c16c2p-10f);
    p = __fadd_rn(__fmul_rn(p, x2), 0x1.555556p-5f);
    p = __fadd_rn(__fmul_rn(p, x2), -0.5f);
    p = __fmul_rn(p, x2);
    return __fadd_rn(1.0f, p);
}
__device__ __forceinline__ float taylor_atan(float z) {  // |z| <= tan(pi/8)
    const float z2 = __fmul_rn(z, z);
    float p = -0x1.642c86p-5f;
    p = __fadd_rn(__fmul_rn(p, z2), 0x1.861862p-5f);
    p = __fadd_rn(__fmul_rn(p, z2), -0x1.af286cp-5f);
    p = __fadd_rn(__fmul_rn(p, z2), 0x1.e1e1e2p-5f);
    p = __fadd_rn(__fmul_rn(p, z2), -0x1.111112p-4f);
    p = __fadd_rn(__fmul_rn(p, z2), 0x1.3b13b2p-4f);
    p = __fadd_rn(__fmul_rn(p, z2), -0x1.745d18p-4f);
    p = __fadd_rn(__fmul_rn(p, z2), 0x1.c71c72p-4f);
    p = __fadd_rn(__fmul_rn(p, z2), -0x1.24924ap-3f);
    p = __fadd_rn(__fmul_rn(p, z2), 0x1.99999ap-3f);
    p = __fadd_rn(__fmul_rn(p, z2), -0x1.555556p-2f);
    p = __fmul_rn(p, z2);
    return __fadd_rn(z, __fmul_rn(z, p));
}
constexpr float kPi4 = 0x1.921fb6p-1f, kPi2 = 0x1.921fb6p+0f, kTwoOverPi = 0x1.45f306p-1f;
constexpr float kTanPi8 = 0x1.a8279ap-2f;
constexpr float kFourPi = 12.566370614359172f;
__device__ __forceinline__ float atan01(float q) {  // q in [0, 1]
    if (q > kTanPi8) {
        const float z = __fdiv_rn(__fsub_rn(q, 1.0f), __fadd_rn(q, 1.0f));
        return __fadd_rn(kPi4, taylor_atan(z));
    }
    return taylor_atan(q);
}

// Concentric octahedral map [-1,1]^2 -> S^2 (Clarberg 2008): diamond rings of
// L1 radius r go to z = 1 - r^2, the azimuth runs linearly along each ring,
// the outer triangles fold onto the lower hemisphere.
__device__ __forceinline__ float3 octa_to_dir(float u, float v) {
    const float au = fabsf(u), av = fabsf(v);
    const float sd = __fsub_rn(1.0f, __fadd_rn(au, av));
    const float r = __fsub_rn(1.0f, fabsf(sd));
    const float phi = (r == 0.0f) ? kPi4
                                  : __fmul_rn(__fadd_rn(__fdiv_rn(__fsub_rn(av, au), r), 1.0f), kPi4);
    const float r2 = __fmul_rn(r, r);
    float z = __fsub_rn(1.0f, r2);
    if (sd < 0.0f) z = -z;
    const float st = __fmul_rn(r, __fsqrt_rn(__fsub_rn(2.0f, r2)));
    float c, s;
    if (phi <= kPi4) {
        c = taylor_cos(phi);
        s = taylor_sin(phi);
    } else {
        const float t = __fsub_rn(kPi2, phi);
        c = taylor_sin(t);
        s = taylor_cos(t);
    }
    const float x = __fmul_rn(c, st), y = __fmul_rn(s, st);
    return make_float3(u < 0.0f ? -x : x, v < 0.0f ? -y : y, z);
}

__device__ __forceinline__ float2 dir_to_octa(float dx, float dy, float dz) {
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    const float r = __fsqrt_rn(__fsub_rn(1.0f, fminf(az, 1.0f)));
    float phi;
    if (ax == 0.0f && ay == 0.0f) phi = 0.0f;
    else if (ay <= ax) phi = atan01(__fdiv_rn(ay, ax));
    else phi = __fsub_rn(kPi2, atan01(__fdiv_rn(ax, ay)));
    const float t = __fmul_rn(phi, kTwoOverPi);
    float bv = __fmul_rn(r, t);
    float bu = __fsub_rn(r, bv);
    if (dz < 0.0f) {
        const float nu = __fsub_rn(1.0f, bv), nv = __fsub_rn(1.0f, bu);
        bu = nu;
        bv = nv;
    }
    return make_float2(dx < 0.0f ? -bu : bu, dy < 0.0f ? -bv : bv);
}

// cell of a direction under the octahedral map (the cell guide_eval_pdf reads)
__device__ __forceinline__ int octa_cell(float3 d, int N) {
    const float2 uv = dir_to_octa(d.x, d.y, d.z);
    const float hn = __fmul_rn((float)N, 0.5f);
    const float a = __fmul_rn(__fadd_rn(uv.x, 1.0f), hn), c = __fmul_rn(__fadd_rn(uv.y, 1.0f), hn);
    const int i = min((a >= 0.0f) ? (int)a : 0, N - 1);
    const int j = min((c >= 0.0f) ? (int)c : 0, N - 1);
    return j * N + i;
}

// cosine-distributed direction about the unit normal n (orthonormal basis of
// Duff et al. 2017, "Building an orthonormal basis, revisited")
__device__ __forceinline__ float3 cosine_dir(float nx, float ny, float nz, float u0, float u1) {
    const float sg = nz >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + nz);
    const float bb = nx * ny * a;
    const float tx = 1.0f + sg * nx * nx * a, ty = sg * bb, tz = -sg * nx;
    const float bx = bb, by = sg + ny * ny * a, bz = -ny;
    const float r = sqrtf(u0);
    float sp, cp;
    sincospif(2.0f * u1, &sp, &cp);
    const float z = sqrtf(fmaxf(0.0f, 1.0f - u0));
    return make_float3(r * cp * tx + r * sp * bx + z * nx, r * cp * ty + r * sp * by + z * ny,
                       r * cp * tz + r * sp * bz + z * nz);
}

// ---------------------------------------------------------------------------
// host-side count of kernel launches issued by this library
void note_launch();
// Reads (and so clears) the last CUDA launch error: WFPG_OK, or WFPG_ERR_CUDA
// with the error remembered for this thread's next error message.
int launch_status();
// The error launch_status() remembered on this thread (cleared), else a fresh
// cudaGetLastError().
cudaError_t take_launch_error();

#define WFPG_LAUNCH(kernel, grid, block, smem, stream, ...)          \
    do {                                                              \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);   \
        ::wfpg::note_launch();                                        \
    } while (0)

__host__ __device__ __forceinline__ uint32_t div_up(uint64_t a, uint64_t b) {
    return (uint32_t)((a + b - 1) / b);
}

}  // namespace wfpg
