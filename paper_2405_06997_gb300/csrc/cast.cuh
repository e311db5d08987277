// Closest-hit ray casting against the procedural scenes' analytic primitives
// (axis-aligned quads, then spheres; a primitive id counts the quads first).
// A renderer-side helper, not part of the guiding method: it moves the
// wavefront from one path vertex to the next.
#pragma once
#include "common.cuh"

namespace wfpg {

struct Hit {
    float t;        // distance along the unit direction, -1 if nothing is hit
    uint32_t prim;  // kNone if nothing is hit
};

__device__ __forceinline__ Hit cast_closest(const float* __restrict__ quads, uint32_t nq,
                                            const float* __restrict__ spheres, uint32_t ns, float ox, float oy,
                                            float oz, float dx, float dy, float dz, float tmin) {
    const float oo[3] = {ox, oy, oz}, dd[3] = {dx, dy, dz};
    float best = __int_as_float(0x7f800000);
    uint32_t bp = kNone;
    for (uint32_t q = 0; q < nq; ++q) {
        const float* Q = quads + 8 * (size_t)q;
        const int a = (int)Q[0], b = (a + 1) % 3, c = (a + 2) % 3;
        if (dd[a] == 0.0f) continue;
        const float t = (Q[1] - oo[a]) / dd[a];
        if (!(t > tmin) || t >= best) continue;
        const float pb = oo[b] + t * dd[b], pc = oo[c] + t * dd[c];
        if (pb >= Q[2] && pb <= Q[3] && pc >= Q[4] && pc <= Q[5]) {
            best = t;
            bp = q;
        }
    }
    for (uint32_t s = 0; s < ns; ++s) {
        const float* S = spheres + 4 * (size_t)s;
        const float cx = ox - S[0], cy = oy - S[1], cz = oz - S[2];
        const float bq = dx * cx + dy * cy + dz * cz;
        const float cq = cx * cx + cy * cy + cz * cz - S[3] * S[3];
        const float disc = bq * bq - cq;
        if (disc < 0.0f) continue;
        const float sq = sqrtf(disc);
        float t = -bq - sq;
        if (!(t > tmin)) t = -bq + sq;
        if (t > tmin && t < best) {
            best = t;
            bp = nq + s;
        }
    }
    return Hit{bp == kNone ? -1.0f : best, bp};
}

// geometric normal at a hit, turned to face the incoming direction d
__device__ __forceinline__ float3 hit_normal(const float* __restrict__ quads, uint32_t nq,
                                             const float* __restrict__ spheres, const Hit& h, float ox, float oy,
                                             float oz, float dx, float dy, float dz) {
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (h.prim != kNone && h.prim < nq) {
        const float* Q = quads + 8 * (size_t)h.prim;
        const int a = (int)Q[0];
        (a == 0 ? nx : (a == 1 ? ny : nz)) = Q[6];
    } else if (h.prim != kNone) {
        const float* S = spheres + 4 * (size_t)(h.prim - nq);
        nx = (ox + h.t * dx - S[0]) / S[3];
        ny = (oy + h.t * dy - S[1]) / S[3];
        nz = (oz + h.t * dz - S[2]) / S[3];
    }
    if (nx * dx + ny * dy + nz * dz > 0.0f) {
        nx = -nx;
        ny = -ny;
        nz = -nz;
    }
    return make_float3(nx, ny, nz);
}

}  // namespace wfpg
