// Closest-hit ray casting against the scenes' primitives (axis-aligned quads,
// spheres, triangles; a primitive id counts the quads, then the spheres, then
// the triangles).  A renderer-side helper, not part of the guiding method: it
// moves the wavefront from one path vertex to the next.
#pragma once
#include "common.cuh"
#include "march.cuh"

namespace wfpg {

struct Hit {
    float t;        // distance along the unit direction, -1 if nothing is hit
    uint32_t prim;  // kNone if nothing is hit
};

// the scene's primitive arrays on the device
struct Prims {
    const float* quads;
    uint32_t nq;
    const float* spheres;
    uint32_t ns;
    const float* tris;
    uint32_t nt;
};

inline Prims prims_of(const wfpg_scene& s) {
    return Prims{s.quads, s.n_quads, s.spheres, s.n_spheres, s.tris, s.n_tris};
}

__device__ __forceinline__ float3 sub3(const float* a, const float* b) {
    return make_float3(a[0] - b[0], a[1] - b[1], a[2] - b[2]);
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// winding normal (v1 - v0) x (v2 - v0) of triangle t, unnormalised
__device__ __forceinline__ float3 tri_cross(const float* T) { return cross3(sub3(T + 3, T), sub3(T + 6, T)); }

// distance to primitive `prim` along the ray (t > tmin), +inf if it is missed;
// triangles by Moller-Trumbore (two-sided)
__device__ __forceinline__ float hit_prim(const Prims& S, uint32_t prim, const float oo[3], const float dd[3],
                                          float tmin) {
    const float INF = __int_as_float(0x7f800000);
    if (prim >= S.nq + S.ns) {
        const float* T = S.tris + 9 * (size_t)(prim - S.nq - S.ns);
        const float3 e1 = sub3(T + 3, T), e2 = sub3(T + 6, T);
        const float3 d = make_float3(dd[0], dd[1], dd[2]);
        const float3 pv = cross3(d, e2);
        const float det = dot3(e1, pv);
        if (det == 0.0f) return INF;
        const float inv = 1.0f / det;
        const float3 tv = make_float3(oo[0] - T[0], oo[1] - T[1], oo[2] - T[2]);
        const float u = dot3(tv, pv) * inv;
        if (!(u >= 0.0f && u <= 1.0f)) return INF;
        const float3 qv = cross3(tv, e1);
        const float v = dot3(d, qv) * inv;
        if (!(v >= 0.0f && u + v <= 1.0f)) return INF;
        const float t = dot3(e2, qv) * inv;
        return t > tmin ? t : INF;
    }
    if (prim < S.nq) {
        const float* Q = S.quads + 8 * (size_t)prim;
        const int a = (int)Q[0], b = (a + 1) % 3, c = (a + 2) % 3;
        if (dd[a] == 0.0f) return INF;
        const float t = (Q[1] - oo[a]) / dd[a];
        if (!(t > tmin)) return INF;
        const float pb = oo[b] + t * dd[b], pc = oo[c] + t * dd[c];
        return (pb >= Q[2] && pb <= Q[3] && pc >= Q[4] && pc <= Q[5]) ? t : INF;
    }
    const float* Sp = S.spheres + 4 * (size_t)(prim - S.nq);
    const float cx = oo[0] - Sp[0], cy = oo[1] - Sp[1], cz = oo[2] - Sp[2];
    const float bq = dd[0] * cx + dd[1] * cy + dd[2] * cz;
    const float cq = cx * cx + cy * cy + cz * cz - Sp[3] * Sp[3];
    const float disc = bq * bq - cq;
    if (disc < 0.0f) return INF;
    const float sq = sqrtf(disc);
    float t = -bq - sq;
    if (!(t > tmin)) t = -bq + sq;
    return t > tmin ? t : INF;
}

// every primitive, nearest first hit (small scenes)
__device__ __forceinline__ Hit cast_closest(const Prims& S, float ox, float oy, float oz, float dx, float dy,
                                            float dz, float tmin) {
    const float oo[3] = {ox, oy, oz}, dd[3] = {dx, dy, dz};
    float best = __int_as_float(0x7f800000);
    uint32_t bp = kNone;
    for (uint32_t p = 0; p < S.nq + S.ns + S.nt; ++p) {
        const float t = hit_prim(S, p, oo, dd, tmin);
        if (t < best) {
            best = t;
            bp = p;
        }
    }
    return Hit{bp == kNone ? -1.0f : best, bp};
}

// The SVO as a ray-casting acceleration structure: node records plus each
// leaf's fragment list (the primitives the conservative voxelisation found in it).
struct SvoCast {
    const Node* node;
    const uint32_t* frag_off;   // per leaf, + 1
    const uint32_t* frag_prim;
    uint32_t leaf_off;          // global id of the first leaf
    int D;
    float lo[3];
    float scale;                // 2^D / S
};

// Closest hit by walking the SVO front to back with the leaf-resolution walk
// of the cone march: every occupied leaf the ray passes is visited in order;
// its primitives are tested and the nearest hit that lies within the leaf's
// stretch of the ray (plus a relative tolerance) ends the walk.  A primitive
// overlaps every leaf its surface passes (conservative voxelisation), so the
// first accepted hit is the closest.  Empty blocks are skipped whole.
__device__ __forceinline__ Hit cast_svo(const SvoCast& V, const Prims& S, float ox, float oy, float oz, float dx,
                                        float dy, float dz, float tmin) {
    const float INF = __int_as_float(0x7f800000);
    const int D = V.D, res = 1 << D;
    const float fres = (float)res;
    const float oo[3] = {ox, oy, oz}, dd[3] = {dx, dy, dz};
    const float gx = (ox - V.lo[0]) * V.scale, gy = (oy - V.lo[1]) * V.scale, gz = (oz - V.lo[2]) * V.scale;
    const float ivx = dx != 0.0f ? 1.0f / (dx * V.scale) : 0.0f;
    const float ivy = dy != 0.0f ? 1.0f / (dy * V.scale) : 0.0f;
    const float ivz = dz != 0.0f ? 1.0f / (dz * V.scale) : 0.0f;
    int cx, cy, cz;
    if (gx >= 0.0f && gx <= fres && gy >= 0.0f && gy <= fres && gz >= 0.0f && gz <= fres) {
        cx = min((int)gx, res - 1);
        cy = min((int)gy, res - 1);
        cz = min((int)gz, res - 1);
    } else {  // slab entry into the grid box
        const float gg[3] = {gx, gy, gz}, iv[3] = {ivx, ivy, ivz};
        float tnr = 0.0f, tfr = INF;
        int enter = -1;
        for (int a = 0; a < 3; ++a) {
            if (iv[a] == 0.0f) {
                if (!(gg[a] >= 0.0f && gg[a] <= fres)) return Hit{-1.0f, kNone};
                continue;
            }
            const float t0 = (0.0f - gg[a]) * iv[a], t1 = (fres - gg[a]) * iv[a];
            const float lo_t = fminf(t0, t1), hi_t = fmaxf(t0, t1);
            if (lo_t > tnr) {
                tnr = lo_t;
                enter = a;
            }
            tfr = fminf(hi_t, tfr);
        }
        if (!(tnr <= tfr)) return Hit{-1.0f, kNone};
        int cc[3];
        for (int a = 0; a < 3; ++a) {
            if (a == enter) {
                cc[a] = iv[a] > 0.0f ? 0 : res - 1;
            } else {
                const float p = gg[a] + tnr * dd[a] * V.scale;
                cc[a] = min((p >= 0.0f) ? (int)p : 0, res - 1);
            }
        }
        cx = cc[0];
        cy = cc[1];
        cz = cc[2];
    }
    uint32_t stk[WFPG_MAX_DEPTH + 1];
    stk[0] = 0;
    int level = 0;
    uint32_t node = 0;
    const int cap = 3 * res + 16;
    for (int steps = 0; steps <= cap; ++steps) {
        while (level < D) {  // deepest existing node holding the cell
            const Node nd = V.node[node];
            const int sh = D - 1 - level;
            const int k = ((cx >> sh) & 1) | (((cy >> sh) & 1) << 1) | (((cz >> sh) & 1) << 2);
            if (!((nd.mask >> k) & 1u)) break;
            node = child_id(nd, k);
            ++level;
            stk[level] = node;
        }
        // exit crossing of the current block (a leaf when level == D)
        const int sl = (level == D) ? 0 : D - level - 1;
        const int size = 1 << sl;
        const int bx = (cx >> sl) << sl, by = (cy >> sl) << sl, bz = (cz >> sl) << sl;
        const int ex = ivx > 0.0f ? bx + size : bx - 1;
        const int ey = ivy > 0.0f ? by + size : by - 1;
        const int ez = ivz > 0.0f ? bz + size : bz - 1;
        const float tex = ivx != 0.0f ? cross_time(ex, ivx > 0.0f, gx, ivx) : INF;
        const float tey = ivy != 0.0f ? cross_time(ey, ivy > 0.0f, gy, ivy) : INF;
        const float tez = ivz != 0.0f ? cross_time(ez, ivz > 0.0f, gz, ivz) : INF;
        const int a = (tex <= tey && tex <= tez) ? 0 : (tey <= tez ? 1 : 2);
        const float tx = a == 0 ? tex : (a == 1 ? tey : tez);
        if (level == D) {
            const uint32_t leaf = node - V.leaf_off;
            float best = INF;
            uint32_t bp = kNone;
            for (uint32_t f = V.frag_off[leaf]; f < V.frag_off[leaf + 1]; ++f) {
                const uint32_t p = V.frag_prim[f];
                const float th = hit_prim(S, p, oo, dd, tmin);
                if (th < best) {
                    best = th;
                    bp = p;
                }
            }
            if (bp != kNone && best <= tx + 1e-5f * fmaxf(1.0f, tx)) return Hit{best, bp};
        }
        // the two other axes p < q by selects: two catch-ups with uniform control flow
        const int p = a == 0 ? 1 : 0, q = a == 2 ? 1 : 2;
        const int np = advance_axis(p == 0 ? cx : cy, p == 0 ? bx : by, size, p == 0 ? gx : gy, p == 0 ? ivx : ivy,
                                    (p == 0 ? dx : dy) * V.scale, tx, p < a);
        const int nq = advance_axis(q == 1 ? cy : cz, q == 1 ? by : bz, size, q == 1 ? gy : gz, q == 1 ? ivy : ivz,
                                    (q == 1 ? dy : dz) * V.scale, tx, q < a);
        const int na = a == 0 ? ex : (a == 1 ? ey : ez);
        const int nx = a == 0 ? na : np;
        const int ny = a == 1 ? na : (p == 1 ? np : nq);
        const int nz = a == 2 ? na : nq;
        if (tx == INF || na < 0 || na >= res) return Hit{-1.0f, kNone};
        const uint32_t diff = (uint32_t)((cx ^ nx) | (cy ^ ny) | (cz ^ nz));
        level = D - 1 - (31 - __clz(diff));
        node = stk[level];
        cx = nx;
        cy = ny;
        cz = nz;
    }
    return Hit{-1.0f, kNone};
}

// geometric normal at a hit, turned to face the incoming direction d
__device__ __forceinline__ float3 hit_normal(const Prims& S, const Hit& h, float ox, float oy, float oz, float dx,
                                             float dy, float dz) {
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (h.prim != kNone && h.prim < S.nq) {
        const float* Q = S.quads + 8 * (size_t)h.prim;
        const int a = (int)Q[0];
        (a == 0 ? nx : (a == 1 ? ny : nz)) = Q[6];
    } else if (h.prim != kNone && h.prim < S.nq + S.ns) {
        const float* Sp = S.spheres + 4 * (size_t)(h.prim - S.nq);
        nx = (ox + h.t * dx - Sp[0]) / Sp[3];
        ny = (oy + h.t * dy - Sp[1]) / Sp[3];
        nz = (oz + h.t * dz - Sp[2]) / Sp[3];
    } else if (h.prim != kNone) {
        const float3 c = tri_cross(S.tris + 9 * (size_t)(h.prim - S.nq - S.ns));
        const float inv = 1.0f / sqrtf(dot3(c, c));
        nx = c.x * inv;
        ny = c.y * inv;
        nz = c.z * inv;
    }
    if (nx * dx + ny * dy + nz * dz > 0.0f) {
        nx = -nx;
        ny = -ny;
        nz = -nz;
    }
    return make_float3(nx, ny, nz);
}

}  // namespace wfpg
