// SVO generation (Sec. 3.2): conservative voxelisation of analytic quads and
// spheres and of triangle meshes (separating-axis test), Morton-key radix sort, unique leaves, level-by-level node
// allocation (children contiguous and Morton-ordered under each parent) and
// two normals per node from k-means with k = 2 (Fig. 2).
#include <string>
#include <vector>

#include "common.cuh"
#include "sort.cuh"
#include "svo.cuh"

namespace wfpg {

constexpr int kPrimBits = 20;  // fragment key = (Morton key << 20) | primitive id

struct PrimRange {
    int lo[3];
    int hi[3];
};

struct SceneDev {
    const float* quads;
    uint32_t nq;
    const float* spheres;
    uint32_t ns;
    const float* tris;
    uint32_t nt;
    float lo[3];
    float S;
    float scale;
    int D;
};

// candidate voxel box of each primitive; quads: exact cells of the closed
// quad; spheres and triangles: bounding box widened by one voxel (the exact
// test decides)
__global__ void k_prim_ranges(SceneDev sc, PrimRange* __restrict__ ranges, uint32_t* __restrict__ cnt,
                              unsigned long long* __restrict__ total, uint32_t* __restrict__ bad) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.nq + sc.ns + sc.nt) return;
    PrimRange r;
    const int res = 1 << sc.D;
    bool ok = true;
    if (p < sc.nq) {
        const float* Q = sc.quads + 8 * (size_t)p;
        const int a = (int)Q[0];
        if (a < 0 || a > 2 || (float)a != Q[0]) {
            ok = false;
            atomicOr(bad, 1u);
        } else {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            r.lo[a] = r.hi[a] = grid_index(Q[1], sc.lo[a], sc.scale, sc.D);
            r.lo[b] = grid_index(Q[2], sc.lo[b], sc.scale, sc.D);
            r.hi[b] = grid_index(Q[3], sc.lo[b], sc.scale, sc.D);
            r.lo[c] = grid_index(Q[4], sc.lo[c], sc.scale, sc.D);
            r.hi[c] = grid_index(Q[5], sc.lo[c], sc.scale, sc.D);
        }
    } else if (p >= sc.nq + sc.ns) {
        const float* T = sc.tris + 9 * (size_t)(p - sc.nq - sc.ns);
        const double h = (double)sc.S / (double)res;
        for (int a = 0; a < 3; ++a) {
            const double mn = fmin((double)T[a], fmin((double)T[3 + a], (double)T[6 + a]));
            const double mx = fmax((double)T[a], fmax((double)T[3 + a], (double)T[6 + a]));
            double l0 = floor(__ddiv_rn(__dsub_rn(mn, (double)sc.lo[a]), h)) - 1.0;
            double l1 = floor(__ddiv_rn(__dsub_rn(mx, (double)sc.lo[a]), h)) + 1.0;
            l0 = fmax(l0, 0.0);
            l1 = fmin(l1, (double)(res - 1));
            r.lo[a] = (int)l0;
            r.hi[a] = (int)l1;
            if (!(l0 <= l1)) ok = false;
        }
    } else {
        const float* P = sc.spheres + 4 * (size_t)(p - sc.nq);
        const double h = (double)sc.S / (double)res;
        for (int a = 0; a < 3; ++a) {
            const double c = P[a], rad = P[3];
            double l0 = floor((c - rad - (double)sc.lo[a]) / h) - 1.0;
            double l1 = floor((c + rad - (double)sc.lo[a]) / h) + 1.0;
            l0 = fmax(l0, 0.0);
            l1 = fmin(l1, (double)(res - 1));
            r.lo[a] = (int)l0;
            r.hi[a] = (int)l1;
            if (!(l0 <= l1)) ok = false;
        }
    }
    uint64_t n = 0;
    if (ok && r.hi[0] >= r.lo[0] && r.hi[1] >= r.lo[1] && r.hi[2] >= r.lo[2])
        n = (uint64_t)(r.hi[0] - r.lo[0] + 1) * (uint64_t)(r.hi[1] - r.lo[1] + 1) *
            (uint64_t)(r.hi[2] - r.lo[2] + 1);
    if (n > 0x7fffffffULL) {
        atomicOr(bad, 2u);
        n = 0;
    }
    if (n == 0) r.lo[0] = r.lo[1] = r.lo[2] = 0, r.hi[0] = r.hi[1] = r.hi[2] = -1;
    ranges[p] = r;
    cnt[p] = (uint32_t)n;
    atomicAdd(total, (unsigned long long)n);
}

// the sphere is voxel-occupying iff min dist(centre, box)^2 <= r^2 <= max dist^2,
// evaluated in binary64 with one rounding per operation
__device__ __forceinline__ bool sphere_hits_voxel(const float* P, const float lo[3], double h, int x,
                                                  int y, int z) {
    const int idx[3] = {x, y, z};
    const double rad = P[3];
    const double r2 = __dmul_rn(rad, rad);
    double dmin2 = 0.0, dmax2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double c = P[a];
        const double bl = __dadd_rn((double)lo[a], __dmul_rn((double)idx[a], h));
        const double bh = __dadd_rn((double)lo[a], __dmul_rn((double)(idx[a] + 1), h));
        const double e = fmax(0.0, fmax(__dsub_rn(bl, c), __dsub_rn(c, bh)));
        dmin2 = __dadd_rn(dmin2, __dmul_rn(e, e));
        const double m = fmax(fabs(__dsub_rn(c, bl)), fabs(__dsub_rn(c, bh)));
        dmax2 = __dadd_rn(dmax2, __dmul_rn(m, m));
    }
    return dmin2 <= r2 && r2 <= dmax2;
}

__device__ __forceinline__ double ddot3(const double a[3], const double b[3]) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

// triangle / closed voxel box overlap by the separating axis theorem
// (Akenine-Moller 2001): disjoint iff the projections separate on one of the
// box's face normals, the triangle's normal, or a box axis crossed with a
// triangle edge.  Box-centred, binary64, one rounding per operation (the
// order fixed, so every caller decides the same voxels); touching overlaps.
__device__ __forceinline__ bool tri_hits_voxel(const float* T, const float lo[3], double h, int x, int y, int z) {
    const int idx[3] = {x, y, z};
    const double e = __dmul_rn(h, 0.5);
    double v[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double c = __dadd_rn((double)lo[a], __dmul_rn(__dadd_rn((double)idx[a], 0.5), h));
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i][a] = __dsub_rn((double)T[3 * i + a], c);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double mn = fmin(v[0][a], fmin(v[1][a], v[2][a]));
        const double mx = fmax(v[0][a], fmax(v[1][a], v[2][a]));
        if (mn > e || mx < -e) return false;
    }
    double f[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) f[i][a] = __dsub_rn(v[(i + 1) % 3][a], v[i][a]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double ax[3];
            ax[k] = 0.0;
            ax[(k + 1) % 3] = -f[i][(k + 2) % 3];
            ax[(k + 2) % 3] = f[i][(k + 1) % 3];
            const double p0 = ddot3(ax, v[0]), p1 = ddot3(ax, v[1]), p2 = ddot3(ax, v[2]);
            const double r = __dmul_rn(e, __dadd_rn(__dadd_rn(fabs(ax[0]), fabs(ax[1])), fabs(ax[2])));
            const double mn = fmin(p0, fmin(p1, p2)), mx = fmax(p0, fmax(p1, p2));
            if (mn > r || mx < -r) return false;
        }
    }
    const double n[3] = {__dsub_rn(__dmul_rn(f[0][1], f[1][2]), __dmul_rn(f[0][2], f[1][1])),
                         __dsub_rn(__dmul_rn(f[0][2], f[1][0]), __dmul_rn(f[0][0], f[1][2])),
                         __dsub_rn(__dmul_rn(f[0][0], f[1][1]), __dmul_rn(f[0][1], f[1][0]))};
    const double d = ddot3(n, v[0]);
    const double r = __dmul_rn(e, __dadd_rn(__dadd_rn(fabs(n[0]), fabs(n[1])), fabs(n[2])));
    return !(d > r || d < -r);
}

template <bool kEmit>
__global__ void __launch_bounds__(256) k_voxel_test(SceneDev sc, const PrimRange* __restrict__ ranges,
                                                    const uint32_t* __restrict__ cand_off, uint32_t n_prims,
                                                    uint32_t total, unsigned long long* __restrict__ counter,
                                                    uint64_t* __restrict__ out, uint32_t out_cap) {
    const int lane = threadIdx.x & 31;
    const double h = (double)sc.S / (double)(1 << sc.D);
    uint32_t local_count = 0;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total;
         base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = base + threadIdx.x;
        bool pass = false;
        uint64_t key = 0;
        if (idx < total) {
            // primitive = last p with cand_off[p] <= idx
            uint32_t lo = 0, hi = n_prims;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (cand_off[mid] <= (uint32_t)idx) lo = mid + 1;
                else hi = mid;
            }
            const uint32_t p = lo - 1;
            const PrimRange r = ranges[p];
            const uint32_t local = (uint32_t)idx - cand_off[p];
            const uint32_t dx = (uint32_t)(r.hi[0] - r.lo[0] + 1), dy = (uint32_t)(r.hi[1] - r.lo[1] + 1);
            const int x = r.lo[0] + (int)(local % dx);
            const int y = r.lo[1] + (int)((local / dx) % dy);
            const int z = r.lo[2] + (int)(local / (dx * dy));
            pass = (p < sc.nq)           ? true
                   : (p < sc.nq + sc.ns) ? sphere_hits_voxel(sc.spheres + 4 * (size_t)(p - sc.nq), sc.lo, h, x, y, z)
                                         : tri_hits_voxel(sc.tris + 9 * (size_t)(p - sc.nq - sc.ns), sc.lo, h, x, y, z);
            key = (morton3((uint32_t)x, (uint32_t)y, (uint32_t)z) << kPrimBits) | p;
        }
        if (kEmit) {
            const uint32_t m = __ballot_sync(0xffffffffu, pass);
            uint32_t slot = 0;
            if (m) {
                const int leader = __ffs(m) - 1;
                if (lane == leader) slot = (uint32_t)atomicAdd(counter, (unsigned long long)__popc(m));
                slot = __shfl_sync(0xffffffffu, slot, leader);
                if (pass) {
                    const uint32_t pos = slot + __popc(m & ((1u << lane) - 1u));
                    if (pos < out_cap) out[pos] = key;
                }
            }
        } else {
            local_count += pass ? 1u : 0u;
        }
    }
    if (!kEmit) {
        for (int k = 16; k > 0; k >>= 1) local_count += __shfl_down_sync(0xffffffffu, local_count, k);
        if (lane == 0 && local_count) atomicAdd(counter, (unsigned long long)local_count);
    }
}

__global__ void k_key_flags(const uint64_t* __restrict__ keys, uint32_t n, int shift, uint32_t* __restrict__ flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift)) ? 1u : 0u;
}

__global__ void k_leaf_compact(const uint64_t* __restrict__ keys, uint32_t n, const uint32_t* __restrict__ flags,
                               const uint32_t* __restrict__ ex, uint64_t* __restrict__ leaf_key,
                               uint32_t* __restrict__ frag_off, uint32_t* __restrict__ frag_prim) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    frag_prim[i] = (uint32_t)(k & ((1u << kPrimBits) - 1u));
    if (flags[i]) {
        leaf_key[ex[i]] = k >> kPrimBits;
        frag_off[ex[i]] = i;
    }
}

// one level up: parent keys = unique(child keys >> 3)
__global__ void k_level_link(const uint64_t* __restrict__ ck, uint32_t nc, const uint32_t* __restrict__ flags,
                             const uint32_t* __restrict__ ex, uint64_t* __restrict__ pk,
                             uint32_t* __restrict__ pfc, uint32_t* __restrict__ cpar) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const uint32_t p = ex[c] + flags[c] - 1u;
    cpar[c] = p;
    if (flags[c]) {
        pk[p] = ck[c] >> 3;
        pfc[p] = c;
    }
}

__global__ void k_level_mask(const uint64_t* __restrict__ ck, uint32_t nc, const uint32_t* __restrict__ pfc,
                             uint32_t np, uint32_t* __restrict__ pmask) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const uint32_t end = (p + 1 < np) ? pfc[p + 1] : nc;
    uint32_t m = 0;
    for (uint32_t c = pfc[p]; c < end; ++c) m |= 1u << (uint32_t)(ck[c] & 7u);
    pmask[p] = m;
}

__global__ void k_assemble_level(uint32_t off, uint32_t n, uint32_t child_off, uint32_t parent_off, int is_leaf,
                                 int is_root, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ fc,
                                 const uint32_t* __restrict__ mask, const uint32_t* __restrict__ par,
                                 Node* __restrict__ node, uint64_t* __restrict__ key, uint32_t* __restrict__ parent) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    Node nd;
    nd.first_child = is_leaf ? kNone : child_off + fc[j];
    nd.mask = is_leaf ? 0u : mask[j];
    node[off + j] = nd;
    key[off + j] = keys[j];
    parent[off + j] = is_root ? kNone : parent_off + par[j];
}

// ---------------------------------------------------------------------------
// k-means, k = 2, over weighted unit vectors supplied by Src::get(f, n, &w):
// centroids start at the first vector and its opposite; four rounds of
// nearest-centroid assignment (squared distance, ties to the first) and
// weighted-mean update (an empty cluster keeps its centroid); the node normal
// is the first centroid normalised (the first vector if that centroid is 0).
template <class Src>
__device__ void kmeans2(const Src& src, int m, float out[3]) {
    float n0[3], w0;
    src.get(0, n0, &w0);
    float c0[3] = {n0[0], n0[1], n0[2]};
    float c1[3] = {-n0[0], -n0[1], -n0[2]};
    for (int it = 0; it < 4; ++it) {
        float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f};
        float k0 = 0.f, k1 = 0.f;
        for (int f = 0; f < m; ++f) {
            float v[3], wf;
            src.get(f, v, &wf);
            const float a0 = __fsub_rn(v[0], c0[0]), a1 = __fsub_rn(v[1], c0[1]), a2 = __fsub_rn(v[2], c0[2]);
            const float b0 = __fsub_rn(v[0], c1[0]), b1 = __fsub_rn(v[1], c1[1]), b2 = __fsub_rn(v[2], c1[2]);
            const float d0 = __fadd_rn(__fadd_rn(__fmul_rn(a0, a0), __fmul_rn(a1, a1)), __fmul_rn(a2, a2));
            const float d1 = __fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2));
            if (d0 <= d1) {
                s0[0] = __fadd_rn(s0[0], __fmul_rn(wf, v[0]));
                s0[1] = __fadd_rn(s0[1], __fmul_rn(wf, v[1]));
                s0[2] = __fadd_rn(s0[2], __fmul_rn(wf, v[2]));
                k0 = __fadd_rn(k0, wf);
            } else {
                s1[0] = __fadd_rn(s1[0], __fmul_rn(wf, v[0]));
                s1[1] = __fadd_rn(s1[1], __fmul_rn(wf, v[1]));
                s1[2] = __fadd_rn(s1[2], __fmul_rn(wf, v[2]));
                k1 = __fadd_rn(k1, wf);
            }
        }
        if (k0 > 0.f) {
            c0[0] = __fdiv_rn(s0[0], k0);
            c0[1] = __fdiv_rn(s0[1], k0);
            c0[2] = __fdiv_rn(s0[2], k0);
        }
        if (k1 > 0.f) {
            c1[0] = __fdiv_rn(s1[0], k1);
            c1[1] = __fdiv_rn(s1[1], k1);
            c1[2] = __fdiv_rn(s1[2], k1);
        }
    }
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(c0[0], c0[0]), __fmul_rn(c0[1], c0[1])), __fmul_rn(c0[2], c0[2]));
    if (len2 > 0.f) {
        const float len = __fsqrt_rn(len2);
        out[0] = __fdiv_rn(c0[0], len);
        out[1] = __fdiv_rn(c0[1], len);
        out[2] = __fdiv_rn(c0[2], len);
    } else {
        out[0] = n0[0];
        out[1] = n0[1];
        out[2] = n0[2];
    }
}

// fragment normals of one leaf: quads give their normal, spheres the unit
// vector from the centre to the voxel centre, triangles their normalised
// winding normal (v1 - v0) x (v2 - v0)
struct LeafFrags {
    const float* quads;
    uint32_t nq;
    const float* spheres;
    uint32_t ns;
    const float* tris;
    const uint32_t* prim;
    float vc[3];
    __device__ void get(int f, float n[3], float* w) const {
        const uint32_t p = prim[f];
        *w = 1.0f;
        if (p >= nq + ns) {
            const float* T = tris + 9 * (size_t)(p - nq - ns);
            const float e1[3] = {__fsub_rn(T[3], T[0]), __fsub_rn(T[4], T[1]), __fsub_rn(T[5], T[2])};
            const float e2[3] = {__fsub_rn(T[6], T[0]), __fsub_rn(T[7], T[1]), __fsub_rn(T[8], T[2])};
            const float c0 = __fsub_rn(__fmul_rn(e1[1], e2[2]), __fmul_rn(e1[2], e2[1]));
            const float c1 = __fsub_rn(__fmul_rn(e1[2], e2[0]), __fmul_rn(e1[0], e2[2]));
            const float c2 = __fsub_rn(__fmul_rn(e1[0], e2[1]), __fmul_rn(e1[1], e2[0]));
            const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(c0, c0), __fmul_rn(c1, c1)), __fmul_rn(c2, c2));
            if (len2 > 0.f) {
                const float len = __fsqrt_rn(len2);
                n[0] = __fdiv_rn(c0, len);
                n[1] = __fdiv_rn(c1, len);
                n[2] = __fdiv_rn(c2, len);
            } else {
                n[0] = 0.f;
                n[1] = 1.f;
                n[2] = 0.f;
            }
            return;
        }
        if (p < nq) {
            const float* Q = quads + 8 * (size_t)p;
            const int a = (int)Q[0];
            n[0] = n[1] = n[2] = 0.0f;
            n[a] = Q[6];
            return;
        }
        const float* P = spheres + 4 * (size_t)(p - nq);
        const float d0 = __fsub_rn(vc[0], P[0]), d1 = __fsub_rn(vc[1], P[1]), d2 = __fsub_rn(vc[2], P[2]);
        const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
        if (len2 > 0.f) {
            const float len = __fsqrt_rn(len2);
            n[0] = __fdiv_rn(d0, len);
            n[1] = __fdiv_rn(d1, len);
            n[2] = __fdiv_rn(d2, len);
        } else {
            n[0] = 0.f;
            n[1] = 1.f;
            n[2] = 0.f;
        }
    }
};

__global__ void k_leaf_normals(SceneDev sc, const uint64_t* __restrict__ leaf_key, uint32_t n_leaves, uint32_t off,
                               const uint32_t* __restrict__ frag_off, const uint32_t* __restrict__ frag_prim,
                               float4* __restrict__ normal, uint32_t* __restrict__ leaf_count) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_leaves) return;
    const uint64_t k = leaf_key[j];
    const uint32_t c[3] = {compact3(k), compact3(k >> 1), compact3(k >> 2)};
    const float h = __fdiv_rn(sc.S, (float)(1 << sc.D));
    LeafFrags src;
    src.quads = sc.quads;
    src.nq = sc.nq;
    src.spheres = sc.spheres;
    src.ns = sc.ns;
    src.tris = sc.tris;
    src.prim = frag_prim + frag_off[j];
    for (int a = 0; a < 3; ++a)
        src.vc[a] = __fadd_rn(sc.lo[a], __fmul_rn(__fadd_rn((float)c[a], 0.5f), h));
    float nrm[3];
    kmeans2(src, (int)(frag_off[j + 1] - frag_off[j]), nrm);
    normal[off + j] = make_float4(nrm[0], nrm[1], nrm[2], 0.0f);
    leaf_count[off + j] = 1u;
}

struct ChildNormals {
    const float4* normal;
    const uint32_t* leaf_count;
    uint32_t first;
    __device__ void get(int f, float n[3], float* w) const {
        const float4 v = normal[first + f];
        n[0] = v.x;
        n[1] = v.y;
        n[2] = v.z;
        *w = __uint2float_rn(leaf_count[first + f]);
    }
};

__global__ void k_inner_normals(uint32_t off, uint32_t n, const Node* __restrict__ node, float4* __restrict__ normal,
                                uint32_t* __restrict__ leaf_count) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const Node nd = node[off + j];
    const int m = __popc(nd.mask);
    ChildNormals src;
    src.normal = normal;
    src.leaf_count = leaf_count;
    src.first = nd.first_child;
    float nrm[3];
    kmeans2(src, m, nrm);
    uint32_t cnt = 0;
    for (int f = 0; f < m; ++f) cnt += leaf_count[nd.first_child + f];
    normal[off + j] = make_float4(nrm[0], nrm[1], nrm[2], 0.0f);
    leaf_count[off + j] = cnt;
}

// ---------------------------------------------------------------------------
namespace {
struct DevBuf {
    void* p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <typename T>
    T* get() { return static_cast<T*>(p); }
};
#define WFPG_TRY(expr)                                        \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) {                              \
            err = std::string(#expr) + ": " + cudaGetErrorString(e_); \
            return WFPG_ERR_CUDA;                             \
        }                                                     \
    } while (0)
#define WFPG_ALLOC(buf, bytes)                                          \
    do {                                                                \
        cudaError_t e_ = cudaMalloc(&(buf), (bytes) != 0 ? (bytes) : 16); \
        if (e_ != cudaSuccess) {                                        \
            err = std::string("device allocation of ") + std::to_string((size_t)(bytes)) + \
                  " bytes failed: " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? WFPG_ERR_OOM : WFPG_ERR_CUDA; \
        }                                                               \
    } while (0)
}  // namespace

// Which parent side each side of a node feeds in the bottom-up average: side s
// of child C (normal (1 - 2s) N_C) goes to the parent's side 0 when
// dot((1 - 2s) N_C, N_P) >= 0, else to side 1.  Fixed once the normals are.
__global__ void k_route(uint32_t n, const uint32_t* __restrict__ parent, const float4* __restrict__ normal,
                        uint8_t* __restrict__ route) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t p = parent[i];
    if (p == kNone) {
        route[i] = 0;
        return;
    }
    const float4 C = normal[i], P = normal[p];
    const float dpos = __fadd_rn(__fadd_rn(__fmul_rn(C.x, P.x), __fmul_rn(C.y, P.y)), __fmul_rn(C.z, P.z));
    const float dneg = __fadd_rn(__fadd_rn(__fmul_rn(-C.x, P.x), __fmul_rn(-C.y, P.y)), __fmul_rn(-C.z, P.z));
    route[i] = (uint8_t)((dpos >= 0.0f ? 0u : 1u) | (dneg >= 0.0f ? 0u : 2u));
}

// One level of the top index: for each cell of level l (row-major, x fastest), the
// deepest existing node at a level <= l containing it, as (level << 28) | node
__global__ void k_top_level(const Node* __restrict__ node, int l, uint32_t* __restrict__ out) {
    const uint32_t R = 1u << l;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * R * R) return;
    const uint32_t x = i & (R - 1), y = (i >> l) & (R - 1), z = i >> (2 * l);
    uint32_t nd = 0;
    int L = 0;
    while (L < l) {
        const Node n = node[nd];
        const int sh = l - 1 - L;
        const int k = (int)(((x >> sh) & 1u) | (((y >> sh) & 1u) << 1) | (((z >> sh) & 1u) << 2));
        if (!((n.mask >> k) & 1u)) break;
        nd = child_id(n, k);
        ++L;
    }
    out[i] = ((uint32_t)L << 28) | nd;
}

// Occupancy bitmap of one level: the bit of each existing node's Morton key
__global__ void k_occ_level(const uint64_t* __restrict__ key, uint32_t first, uint32_t count,
                            uint32_t* __restrict__ bits) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t k = key[first + i];
    atomicOr(&bits[k >> 5], 1u << (uint32_t)(k & 31u));
}

void svo_free_arrays(wfpg_svo* s) {
    void* ptrs[] = {s->node, s->parent, s->key, s->leaf_count, s->normal, s->route, s->frag_off, s->frag_prim,
                    s->acc_sum, s->acc_cnt, s->tot_sum, s->tot_cnt, s->value, s->status, s->top, s->occ};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

int build_svo(const wfpg_scene* scene, int D, cudaStream_t st, wfpg_svo* s, std::string& err) {
    SceneDev sc;
    sc.quads = scene->quads;
    sc.nq = scene->n_quads;
    sc.spheres = scene->spheres;
    sc.ns = scene->n_spheres;
    sc.tris = scene->tris;
    sc.nt = scene->n_tris;
    for (int a = 0; a < 3; ++a) sc.lo[a] = scene->lo[a];
    sc.S = scene->size;
    sc.scale = (float)(1 << D) / scene->size;
    sc.D = D;
    s->D = D;
    for (int a = 0; a < 3; ++a) s->lo[a] = sc.lo[a];
    s->S = sc.S;
    s->scale = sc.scale;
    const uint32_t n_prims = sc.nq + sc.ns + sc.nt;
    const int T = 256;

    // 1. candidate boxes and counts
    DevBuf ranges, cnt, misc, ws_buf;
    WFPG_ALLOC(ranges.p, sizeof(PrimRange) * n_prims);
    WFPG_ALLOC(cnt.p, 4 * (size_t)n_prims + 4);
    WFPG_ALLOC(misc.p, 64);
    unsigned long long* total = misc.get<unsigned long long>();
    uint32_t* bad = reinterpret_cast<uint32_t*>(misc.get<char>() + 8);
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(misc.get<char>() + 16);
    uint32_t* dev_total32 = reinterpret_cast<uint32_t*>(misc.get<char>() + 24);
    WFPG_TRY(cudaMemsetAsync(misc.p, 0, 64, st));
    WFPG_LAUNCH(k_prim_ranges, div_up(n_prims, T), T, 0, st, sc, ranges.get<PrimRange>(), cnt.get<uint32_t>(), total, bad);
    unsigned long long h_total = 0;
    uint32_t h_bad = 0;
    WFPG_TRY(cudaMemcpyAsync(&h_total, total, 8, cudaMemcpyDeviceToHost, st));
    WFPG_TRY(cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, st));
    WFPG_TRY(cudaStreamSynchronize(st));
    if (h_bad & 1u) { err = "a quad's axis is not 0, 1 or 2"; return WFPG_ERR_INVALID_ARG; }
    if (h_bad & 2u) { err = "a primitive spans more than 2^31 candidate voxels"; return WFPG_ERR_INVALID_ARG; }
    if (h_total >= 0xffffffffULL) { err = "more than 2^32 candidate voxels"; return WFPG_ERR_INVALID_ARG; }
    const uint32_t n_cand = (uint32_t)h_total;
    if (n_cand == 0) { err = "the scene occupies no voxel"; return WFPG_ERR_INVALID_ARG; }

    size_t ws_bytes = scan_workspace_bytes(n_prims) + (64u << 20);
    WFPG_ALLOC(ws_buf.p, ws_bytes);
    Arena ws{ws_buf.get<char>(), ws_bytes, 0, false};
    scan_exclusive(cnt.get<uint32_t>(), cnt.get<uint32_t>(), n_prims, nullptr, ws, st);
    ws.used = 0;

    // 2. count and emit fragments (key << 20 | prim)
    const uint32_t grid = 152 * 8;
    WFPG_LAUNCH(k_voxel_test<false>, grid, T, 0, st, sc, ranges.get<PrimRange>(), cnt.get<uint32_t>(), n_prims, n_cand,
                                            counter, nullptr, 0);
    unsigned long long h_frags = 0;
    WFPG_TRY(cudaMemcpyAsync(&h_frags, counter, 8, cudaMemcpyDeviceToHost, st));
    WFPG_TRY(cudaStreamSynchronize(st));
    if (h_frags == 0) { err = "the scene occupies no voxel"; return WFPG_ERR_INVALID_ARG; }
    if (h_frags >= 0x7fffffffULL) { err = "more than 2^31 voxel fragments"; return WFPG_ERR_INVALID_ARG; }
    const uint32_t nf = (uint32_t)h_frags;
    DevBuf fk, fk_alt;
    WFPG_ALLOC(fk.p, 8 * (size_t)nf);
    WFPG_ALLOC(fk_alt.p, 8 * (size_t)nf);
    WFPG_TRY(cudaMemsetAsync(counter, 0, 8, st));
    WFPG_LAUNCH(k_voxel_test<true>, grid, T, 0, st, sc, ranges.get<PrimRange>(), cnt.get<uint32_t>(), n_prims, n_cand,
                                           counter, fk.get<uint64_t>(), nf);

    // 3. sort fragments
    size_t need = radix_sort_workspace_bytes(nf) + 3 * arena_bytes<uint32_t>(nf) + scan_workspace_bytes(nf);
    if (need > ws_bytes) {
        cudaFree(ws_buf.p);
        ws_buf.p = nullptr;
        ws_bytes = need;
        WFPG_ALLOC(ws_buf.p, ws_bytes);
        ws = Arena{ws_buf.get<char>(), ws_bytes, 0, false};
    }
    uint64_t* sorted = nullptr;
    radix_sort_u64(fk.get<uint64_t>(), fk_alt.get<uint64_t>(), nf, 3 * D + kPrimBits, ws, st, &sorted);
    ws.used = 0;

    // 4. unique leaves and fragment lists
    uint32_t* flags = ws.take<uint32_t>(nf);
    uint32_t* ex = ws.take<uint32_t>(nf);
    WFPG_LAUNCH(k_key_flags, div_up(nf, T), T, 0, st, sorted, nf, kPrimBits, flags);
    scan_exclusive(flags, ex, nf, dev_total32, ws, st);
    uint32_t n_leaves = 0;
    WFPG_TRY(cudaMemcpyAsync(&n_leaves, dev_total32, 4, cudaMemcpyDeviceToHost, st));
    WFPG_TRY(cudaStreamSynchronize(st));
    WFPG_ALLOC(s->frag_off, 4 * ((size_t)n_leaves + 1));
    WFPG_ALLOC(s->frag_prim, 4 * (size_t)nf);
    std::vector<DevBuf> lkeys(D + 1), lfc(D + 1), lmask(D + 1), lpar(D + 1);
    std::vector<uint32_t> lsize(D + 1, 0);
    WFPG_ALLOC(lkeys[D].p, 8 * (size_t)n_leaves);
    WFPG_LAUNCH(k_leaf_compact, div_up(nf, T), T, 0, st, sorted, nf, flags, ex, lkeys[D].get<uint64_t>(), s->frag_off,
                                                s->frag_prim);
    WFPG_TRY(cudaMemcpyAsync(s->frag_off + n_leaves, &nf, 4, cudaMemcpyHostToDevice, st));
    lsize[D] = n_leaves;
    s->n_frags = nf;

    // 5. levels D-1 .. 0
    for (int l = D - 1; l >= 0; --l) {
        const uint32_t nc = lsize[l + 1];
        ws.used = 0;
        uint32_t* fl = ws.take<uint32_t>(nc);
        uint32_t* e2 = ws.take<uint32_t>(nc);
        const uint64_t* ck = lkeys[l + 1].get<uint64_t>();
        WFPG_LAUNCH(k_key_flags, div_up(nc, T), T, 0, st, ck, nc, 3, fl);
        scan_exclusive(fl, e2, nc, dev_total32, ws, st);
        uint32_t np = 0;
        WFPG_TRY(cudaMemcpyAsync(&np, dev_total32, 4, cudaMemcpyDeviceToHost, st));
        WFPG_TRY(cudaStreamSynchronize(st));
        lsize[l] = np;
        WFPG_ALLOC(lkeys[l].p, 8 * (size_t)np);
        WFPG_ALLOC(lfc[l].p, 4 * (size_t)np);
        WFPG_ALLOC(lmask[l].p, 4 * (size_t)np);
        WFPG_ALLOC(lpar[l + 1].p, 4 * (size_t)nc);
        WFPG_LAUNCH(k_level_link, div_up(nc, T), T, 0, st, ck, nc, fl, e2, lkeys[l].get<uint64_t>(), lfc[l].get<uint32_t>(),
                                                  lpar[l + 1].get<uint32_t>());
        WFPG_LAUNCH(k_level_mask, div_up(np, T), T, 0, st, ck, nc, lfc[l].get<uint32_t>(), np, lmask[l].get<uint32_t>());
    }
    s->level_off[0] = 0;
    for (int l = 0; l <= D; ++l) s->level_off[l + 1] = s->level_off[l] + lsize[l];
    for (int l = D + 2; l < WFPG_MAX_DEPTH + 2; ++l) s->level_off[l] = s->level_off[D + 1];
    const uint32_t nn = s->level_off[D + 1];
    s->n_nodes = nn;

    // 6. global arrays
    WFPG_ALLOC(s->node, sizeof(Node) * (size_t)nn);
    WFPG_ALLOC(s->parent, 4 * (size_t)nn);
    WFPG_ALLOC(s->key, 8 * (size_t)nn);
    WFPG_ALLOC(s->leaf_count, 4 * (size_t)nn);
    WFPG_ALLOC(s->normal, sizeof(float4) * (size_t)nn);
    for (int l = 0; l <= D; ++l) {
        const uint32_t n = lsize[l];
        WFPG_LAUNCH(k_assemble_level, div_up(n, T), T, 0, st, 
            s->level_off[l], n, l < D ? s->level_off[l + 1] : 0u, l > 0 ? s->level_off[l - 1] : 0u, l == D, l == 0,
            lkeys[l].get<uint64_t>(), l < D ? lfc[l].get<uint32_t>() : nullptr,
            l < D ? lmask[l].get<uint32_t>() : nullptr, l > 0 ? lpar[l].get<uint32_t>() : nullptr, s->node, s->key,
            s->parent);
    }
    // 7. normals, leaves then levels upward
    WFPG_LAUNCH(k_leaf_normals, div_up(n_leaves, T), T, 0, st, sc, lkeys[D].get<uint64_t>(), n_leaves, s->level_off[D],
                                                      s->frag_off, s->frag_prim, s->normal, s->leaf_count);
    for (int l = D - 1; l >= 0; --l)
        WFPG_LAUNCH(k_inner_normals, div_up(lsize[l], T), T, 0, st, s->level_off[l], lsize[l], s->node, s->normal,
                                                           s->leaf_count);
    WFPG_ALLOC(s->route, (size_t)nn);
    WFPG_LAUNCH(k_route, div_up(nn, T), T, 0, st, nn, s->parent, s->normal, s->route);
    // 8. the top index of levels 0 .. min(D, kTopLevelMax) (node ids must fit in 28 bits)
    if (nn < (1u << 28)) {
        const int G = D < kTopLevelMax ? D : kTopLevelMax;
        size_t cells = 0;
        for (int l = 0; l <= G; ++l) {
            s->top_off[l] = (uint32_t)cells;
            cells += (size_t)1 << (3 * l);
        }
        WFPG_ALLOC(s->top, sizeof(uint32_t) * cells);
        for (int l = 0; l <= G; ++l)
            WFPG_LAUNCH(k_top_level, div_up((size_t)1 << (3 * l), T), T, 0, st, s->node, l, s->top + s->top_off[l]);
        s->top_levels = G + 1;
        // occupancy bitmaps of the levels below the index (levels > 6 hold 8^l >= 2^21 bits)
        if (D > G && D <= kOccMaxDepth) {
            const uint64_t words = occ_offset(G, D + 1);
            WFPG_ALLOC(s->occ, sizeof(uint32_t) * words);
            WFPG_TRY(cudaMemsetAsync(s->occ, 0, sizeof(uint32_t) * words, st));
            for (int l = G + 1; l <= D; ++l) {
                s->occ_off[l] = occ_offset(G, l);
                const uint32_t cnt = s->level_off[l + 1] - s->level_off[l];
                WFPG_LAUNCH(k_occ_level, div_up(cnt, T), T, 0, st, s->key, s->level_off[l], cnt, s->occ + s->occ_off[l]);
            }
        }
    }
    // 9. exitance arrays, zeroed
    WFPG_ALLOC(s->acc_sum, 16 * (size_t)nn);
    WFPG_ALLOC(s->tot_sum, 16 * (size_t)nn);
    WFPG_ALLOC(s->acc_cnt, 8 * (size_t)nn);
    WFPG_ALLOC(s->tot_cnt, 8 * (size_t)nn);
    WFPG_ALLOC(s->value, sizeof(float2) * (size_t)nn);
    WFPG_ALLOC(s->status, 16);
    s->bin_next = s->status + 1;
    WFPG_TRY(cudaMemsetAsync(s->acc_sum, 0, 16 * (size_t)nn, st));
    WFPG_TRY(cudaMemsetAsync(s->tot_sum, 0, 16 * (size_t)nn, st));
    WFPG_TRY(cudaMemsetAsync(s->acc_cnt, 0, 8 * (size_t)nn, st));
    WFPG_TRY(cudaMemsetAsync(s->tot_cnt, 0, 8 * (size_t)nn, st));
    WFPG_TRY(cudaMemsetAsync(s->value, 0, sizeof(float2) * (size_t)nn, st));
    WFPG_TRY(cudaMemsetAsync(s->status, 0, 16, st));
    WFPG_TRY(cudaGetLastError());
    WFPG_TRY(cudaStreamSynchronize(st));
    return WFPG_OK;
}

}  // namespace wfpg
