// CPU ORACLE -- TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
//
// Directions and cone queries (Sec. 3.3 and Sec. 3 "Implementation"):
//  * own sine, cosine and arctangent (Taylor series, stated below), so that
//    the map from grid cells to directions does not depend on a math library;
//  * the concentric octahedral map of Clarberg (2008), which the paper uses to
//    lay the directional radiance field on a 2D grid of equal-solid-angle
//    cells;
//  * ConeTrace: the first occupied leaf along the ray (a leaf-resolution 3D
//    DDA after Amanatides & Woo 1987 -- the paper finds the hit with hardware
//    ray tracing), then the ancestor whose squared side is closest to the cone
//    footprint A = r^2 * omega (Eq. 6), then that node's exitance on the side
//    facing the query point.
#include <algorithm>
#include <cmath>
#include <limits>

#include "oracle_internal.h"

namespace orc {

// sin x = sum_k (-1)^k x^(2k+1) / (2k+1)!   for |x| <= pi/4, terms to x^11
float poly_sin(float x) {
    float x2 = x * x;
    float p = -0x1.ae6456p-26f;          // -1/11!
    p = p * x2 + 0x1.71de3ap-19f;        //  1/9!
    p = p * x2 + -0x1.a01a02p-13f;       // -1/7!
    p = p * x2 + 0x1.111112p-7f;         //  1/5!
    p = p * x2 + -0x1.555556p-3f;        // -1/3!
    p = p * x2;
    return x + x * p;
}

// cos x = sum_k (-1)^k x^(2k) / (2k)!   for |x| <= pi/4, terms to x^10
float poly_cos(float x) {
    float x2 = x * x;
    float p = -0x1.27e4fcp-22f;          // -1/10!
    p = p * x2 + 0x1.a01a02p-16f;        //  1/8!
    p = p * x2 + -0x1.6c16c2p-10f;       // -1/6!
    p = p * x2 + 0x1.555556p-5f;         //  1/4!
    p = p * x2 + -0.5f;                  // -1/2!
    p = p * x2;
    return 1.0f + p;
}

// atan z = sum_k (-1)^k z^(2k+1) / (2k+1)   for |z| <= tan(pi/8), terms to z^23
static float atan_series(float z) {
    float z2 = z * z;
    float p = -0x1.642c86p-5f;           // -1/23
    p = p * z2 + 0x1.861862p-5f;         //  1/21
    p = p * z2 + -0x1.af286cp-5f;        // -1/19
    p = p * z2 + 0x1.e1e1e2p-5f;         //  1/17
    p = p * z2 + -0x1.111112p-4f;        // -1/15
    p = p * z2 + 0x1.3b13b2p-4f;         //  1/13
    p = p * z2 + -0x1.745d18p-4f;        // -1/11
    p = p * z2 + 0x1.c71c72p-4f;         //  1/9
    p = p * z2 + -0x1.24924ap-3f;        // -1/7
    p = p * z2 + 0x1.99999ap-3f;         //  1/5
    p = p * z2 + -0x1.555556p-2f;        // -1/3
    p = p * z2;
    return z + z * p;
}

// atan q for q in [0, 1]; above tan(pi/8) use atan q = pi/4 + atan((q-1)/(q+1))
float poly_atan01(float q) {
    if (q > 0x1.a8279ap-2f) {
        float z = (q - 1.0f) / (q + 1.0f);
        return 0x1.921fb6p-1f + atan_series(z);
    }
    return atan_series(q);
}

static constexpr float PI_4 = 0x1.921fb6p-1f;
static constexpr float PI_2 = 0x1.921fb6p+0f;
static constexpr float TWO_OVER_PI = 0x1.45f306p-1f;

// Concentric octahedral map, square [-1,1]^2 -> unit sphere (Clarberg 2008).
// The diamond |u|+|v| <= 1 is the upper hemisphere; each diamond ring of L1
// radius r maps to the circle z = 1 - r^2 (equal area: the diamond of radius
// r covers 2 r^2 of the square's 4, the cap 2 pi (1 - z) of the sphere's
// 4 pi), and the azimuth is linear along the ring.  The outer triangles fold
// onto the lower hemisphere.
void octa_decode(float u, float v, float out[3]) {
    float au = std::fabs(u), av = std::fabs(v);
    float sd = 1.0f - (au + av);
    float r = 1.0f - std::fabs(sd);
    float phi = (r == 0.0f) ? PI_4 : ((av - au) / r + 1.0f) * PI_4;
    float r2 = r * r;
    float z = 1.0f - r2;
    if (sd < 0.0f) z = -z;
    float st = r * std::sqrt(2.0f - r2);
    float c, s;
    if (phi <= PI_4) {
        c = poly_cos(phi);
        s = poly_sin(phi);
    } else {
        float t = PI_2 - phi;
        c = poly_sin(t);
        s = poly_cos(t);
    }
    float x = c * st, y = s * st;
    out[0] = (u < 0.0f) ? -x : x;
    out[1] = (v < 0.0f) ? -y : y;
    out[2] = z;
}

// inverse of octa_decode
void octa_encode(const float d[3], float* u, float* v) {
    float ax = std::fabs(d[0]), ay = std::fabs(d[1]), az = std::fabs(d[2]);
    float r = std::sqrt(1.0f - std::min(az, 1.0f));
    float phi;
    if (ax == 0.0f && ay == 0.0f) phi = 0.0f;
    else if (ay <= ax) phi = poly_atan01(ay / ax);
    else phi = PI_2 - poly_atan01(ax / ay);
    float t = phi * TWO_OVER_PI;
    float bv = r * t;
    float bu = r - bv;
    if (d[2] < 0.0f) {
        float nu = 1.0f - bv, nv = 1.0f - bu;
        bu = nu;
        bv = nv;
    }
    *u = (d[0] < 0.0f) ? -bu : bu;
    *v = (d[1] < 0.0f) ? -bv : bv;
}

// ---------------------------------------------------------------------------
// ConeTrace for one grid cell (Sec. 3.3, Eq. 6).
// The ray o + t d walks the leaf grid cell by cell (Amanatides & Woo).  Every
// boundary time is evaluated afresh as t = (k - g_a) / (d_a * 2^D / S) for
// the integer boundary k, never accumulated; the next axis is the one with
// the smallest time, ties in the order x, y, z.  The answer is the first
// occupied leaf entered at t >= t_skip (reading: t_skip stands in for the
// paper's ray offset at the origin's own surface).
TraceResult trace_cell(const Svo& s, const float o[3], const float d[3], float t_skip,
                       float omega, int cos_weight, bool count_blocks) {
    TraceResult R{};
    R.hit = 0;
    R.value = 0.0f;
    R.node = NONE;
    const int D = s.D;
    const int32_t res = 1 << D;
    const float fres = (float)res;
    const float INF = std::numeric_limits<float>::infinity();
    float g[3], inv[3], dsc[3];
    int step[3];
    bool moving[3];
    for (int a = 0; a < 3; ++a) {
        g[a] = (o[a] - s.lo[a]) * s.scale;
        dsc[a] = d[a] * s.scale;
        moving[a] = d[a] != 0.0f;
        inv[a] = moving[a] ? 1.0f / dsc[a] : 0.0f;
        step[a] = d[a] > 0.0f ? 1 : -1;
    }
    int32_t cell[3];
    float t_cur = 0.0f;
    bool inside = true;
    for (int a = 0; a < 3; ++a) inside = inside && (g[a] >= 0.0f) && (g[a] <= fres);
    if (inside) {
        for (int a = 0; a < 3; ++a) cell[a] = std::min((int32_t)g[a], res - 1);
    } else {
        // slab entry into the grid box
        float tn = 0.0f, tf = INF;
        int enter_axis = -1;
        for (int a = 0; a < 3; ++a) {
            if (!moving[a]) {
                if (!(g[a] >= 0.0f && g[a] <= fres)) return R;
                continue;
            }
            float t0 = (0.0f - g[a]) * inv[a];
            float t1 = (fres - g[a]) * inv[a];
            float lo_t = std::min(t0, t1), hi_t = std::max(t0, t1);
            if (lo_t > tn) { tn = lo_t; enter_axis = a; }
            tf = std::min(tf, hi_t);
        }
        if (!(tn <= tf)) return R;
        t_cur = tn;
        for (int a = 0; a < 3; ++a) {
            if (a == enter_axis) {
                cell[a] = step[a] > 0 ? 0 : res - 1;
            } else {
                float p = g[a] + tn * dsc[a];
                int32_t c = (p >= 0.0f) ? (int32_t)p : 0;
                cell[a] = std::min(c, res - 1);
            }
        }
    }
    uint32_t steps = 0, blocks = 0;
    int prev_level = -1;
    uint64_t prev_block = 0;
    for (;;) {
        ++steps;
        uint64_t key = morton((uint32_t)cell[0], (uint32_t)cell[1], (uint32_t)cell[2]);
        if (count_blocks) {
            // instrumentation: the largest block holding this cell that is
            // either one occupied leaf or empty (the child of the deepest
            // existing ancestor); count each new block the ray enters
            int L = D;
            while (L > 0 && s.find(L, key >> (3 * (D - L))) == NONE) --L;
            int bl = (L == D) ? D : L + 1;
            uint64_t b = key >> (3 * (D - bl));
            if (bl != prev_level || b != prev_block) ++blocks;
            prev_level = bl;
            prev_block = b;
        }
        if (t_cur >= t_skip && s.find(D, key) != NONE) {
            R.hit = 1;
            R.leaf_key = key;
            R.t_entry = t_cur;
            break;
        }
        float tn[3];
        for (int a = 0; a < 3; ++a) {
            if (!moving[a]) { tn[a] = INF; continue; }
            int32_t k = step[a] > 0 ? cell[a] + 1 : cell[a];
            tn[a] = ((float)k - g[a]) * inv[a];
        }
        int a = (tn[0] <= tn[1] && tn[0] <= tn[2]) ? 0 : (tn[1] <= tn[2] ? 1 : 2);
        if (tn[a] == INF) break;
        t_cur = tn[a];
        cell[a] += step[a];
        if (cell[a] < 0 || cell[a] >= res) break;
    }
    R.steps = steps;
    R.blocks = blocks;
    if (!R.hit) return R;
    // Eq. 6: footprint A = r^2 * omega with r the entry distance; choose the
    // level whose squared node side is closest to A (ties to the finer level)
    float A = (R.t_entry * R.t_entry) * omega;
    float side = s.S;
    int best = 0;
    float best_diff = INF;
    for (int l = 0; l <= D; ++l) {
        float diff = std::fabs(side * side - A);
        if (diff <= best_diff) {
            best_diff = diff;
            best = l;
        }
        side = side * 0.5f;
    }
    R.level = best;
    R.node = s.find(best, R.leaf_key >> (3 * (D - best)));
    // Reading of "multiplying the voxel normal with the cone's principal
    // direction": take the side whose normal faces back along the cone
    // (dot(N, -d) >= 0 -> side 0).
    const float* N = &s.normal[3 * (size_t)R.node];
    float dd = N[0] * d[0] + N[1] * d[1] + N[2] * d[2];
    R.side = (dd <= 0.0f) ? 0 : 1;
    R.value = s.value[2 * (size_t)R.node + R.side];
    if (cos_weight) R.value = R.value * std::fabs(dd);
    return R;
}

}  // namespace orc
