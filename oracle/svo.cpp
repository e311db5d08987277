// CPU ORACLE -- TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
//
// SVO construction and radiant-exitance caching, Sec. 3.2 of the paper:
//  * conservative voxelisation of the scene (the paper rasterises triangles,
//    after Crassin & Green 2012; here analytic quads and spheres, and
//    triangles by the separating-axis test, against closed voxel boxes),
//  * Morton-key sort and a level-by-level unique-prefix hierarchy (the paper
//    builds it after Karras 2012; the set of octree nodes is the same),
//  * two normals per node from k-means with k = 2 (Fig. 2),
//  * UpdateExitance: each path-vertex record is added to the leaf holding it
//    (Eq. 5 and Alg. 1), and the leaf values are averaged bottom-up.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "oracle_internal.h"

namespace orc {

uint32_t Svo::find(int l, uint64_t prefix) const {
    const std::vector<uint64_t>& k = keys[l];
    auto it = std::lower_bound(k.begin(), k.end(), prefix);
    if (it == k.end() || *it != prefix) return NONE;
    return level_off[l] + (uint32_t)(it - k.begin());
}

uint32_t Svo::deepest(const float p[3]) const {
    uint32_t ix = (uint32_t)grid_index(p[0], lo[0], scale, D);
    uint32_t iy = (uint32_t)grid_index(p[1], lo[1], scale, D);
    uint32_t iz = (uint32_t)grid_index(p[2], lo[2], scale, D);
    uint64_t key = morton(ix, iy, iz);
    for (int l = D; l >= 0; --l) {
        uint32_t n = find(l, key >> (3 * (D - l)));
        if (n != NONE) return n;
    }
    return NONE;
}

// ---------------------------------------------------------------------------
// k-means, k = 2, on unit vectors n[m] with weights w[m] (Sec. 3.2, Fig. 2).
// Reading of the paper: the first centroid starts at the first element (the
// paper draws a random surface element; the lowest primitive index is used
// so that the result is reproducible), the second at its opposite; four
// rounds of nearest-centroid assignment (squared distance, ties to the first
// centroid) and weighted-mean update; an empty cluster keeps its centroid.
// The node normal N is the first centroid normalised (the first element if
// the centroid is the zero vector); the node's second normal is -N.
void kmeans2(const float* n, const float* w, int m, float out[3]) {
    float c0[3] = {n[0], n[1], n[2]};
    float c1[3] = {-n[0], -n[1], -n[2]};
    for (int it = 0; it < 4; ++it) {
        float s0[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
        float k0 = 0, k1 = 0;
        for (int f = 0; f < m; ++f) {
            const float* v = n + 3 * f;
            float a0 = v[0] - c0[0], a1 = v[1] - c0[1], a2 = v[2] - c0[2];
            float b0 = v[0] - c1[0], b1 = v[1] - c1[1], b2 = v[2] - c1[2];
            float d0 = a0 * a0 + a1 * a1 + a2 * a2;
            float d1 = b0 * b0 + b1 * b1 + b2 * b2;
            float wf = w[f];
            if (d0 <= d1) {
                s0[0] = s0[0] + wf * v[0];
                s0[1] = s0[1] + wf * v[1];
                s0[2] = s0[2] + wf * v[2];
                k0 = k0 + wf;
            } else {
                s1[0] = s1[0] + wf * v[0];
                s1[1] = s1[1] + wf * v[1];
                s1[2] = s1[2] + wf * v[2];
                k1 = k1 + wf;
            }
        }
        if (k0 > 0) { c0[0] = s0[0] / k0; c0[1] = s0[1] / k0; c0[2] = s0[2] / k0; }
        if (k1 > 0) { c1[0] = s1[0] / k1; c1[1] = s1[1] / k1; c1[2] = s1[2] / k1; }
    }
    float len2 = c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2];
    if (len2 > 0) {
        float len = std::sqrt(len2);
        out[0] = c0[0] / len;
        out[1] = c0[1] / len;
        out[2] = c0[2] / len;
    } else {
        out[0] = n[0];
        out[1] = n[1];
        out[2] = n[2];
    }
}

namespace {

struct Frag {
    uint64_t key;
    uint32_t prim;
    bool operator<(const Frag& o) const {
        return key != o.key ? key < o.key : prim < o.prim;
    }
};

double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Triangle / closed box overlap by the separating axis theorem (Akenine-Moller
// 2001): the two convex sets are disjoint iff their projections are disjoint on
// one of 13 axes -- the box's three face normals, the triangle's normal, and
// the nine cross products of a box axis with a triangle edge.  Box-centred
// coordinates, binary64, one rounding per written operation; touching counts
// as overlap.
bool tri_box_overlap(const float* T, const double c[3], double e) {
    double v[3][3];
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) v[i][a] = (double)T[3 * i + a] - c[a];
    for (int a = 0; a < 3; ++a) {  // face normals: the triangle's bounding interval against [-e, e]
        double mn = std::min(v[0][a], std::min(v[1][a], v[2][a]));
        double mx = std::max(v[0][a], std::max(v[1][a], v[2][a]));
        if (mn > e || mx < -e) return false;
    }
    double f[3][3];  // edges v1 - v0, v2 - v1, v0 - v2
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) f[i][a] = v[(i + 1) % 3][a] - v[i][a];
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) {  // axis e_k x f_i
            double ax[3];
            ax[k] = 0.0;
            ax[(k + 1) % 3] = -f[i][(k + 2) % 3];
            ax[(k + 2) % 3] = f[i][(k + 1) % 3];
            double p0 = dot3(ax, v[0]), p1 = dot3(ax, v[1]), p2 = dot3(ax, v[2]);
            double r = e * (std::fabs(ax[0]) + std::fabs(ax[1]) + std::fabs(ax[2]));
            double mn = std::min(p0, std::min(p1, p2)), mx = std::max(p0, std::max(p1, p2));
            if (mn > r || mx < -r) return false;
        }
    }
    // the triangle's plane
    double n[3] = {f[0][1] * f[1][2] - f[0][2] * f[1][1], f[0][2] * f[1][0] - f[0][0] * f[1][2],
                   f[0][0] * f[1][1] - f[0][1] * f[1][0]};
    double d = dot3(n, v[0]);
    double r = e * (std::fabs(n[0]) + std::fabs(n[1]) + std::fabs(n[2]));
    return !(d > r || d < -r);
}

// Conservative voxelisation: a voxel is occupied when the primitive's surface
// meets the closed voxel box.
void voxelize(const float* quads, int nq, const float* spheres, int ns, const float* tris, int nt,
              const float lo[3], float S, int D, std::vector<Frag>& out) {
    const float scale = (float)(1 << D) / S;
    for (int q = 0; q < nq; ++q) {
        const float* Q = quads + 8 * q;
        int a = (int)Q[0], b = (a + 1) % 3, c = (a + 2) % 3;
        int layer = grid_index(Q[1], lo[a], scale, D);
        int b0 = grid_index(Q[2], lo[b], scale, D), b1 = grid_index(Q[3], lo[b], scale, D);
        int c0 = grid_index(Q[4], lo[c], scale, D), c1 = grid_index(Q[5], lo[c], scale, D);
        for (int ib = b0; ib <= b1; ++ib)
            for (int ic = c0; ic <= c1; ++ic) {
                uint32_t x[3];
                x[a] = (uint32_t)layer;
                x[b] = (uint32_t)ib;
                x[c] = (uint32_t)ic;
                out.push_back({morton(x[0], x[1], x[2]), (uint32_t)q});
            }
    }
    // spheres: occupied iff min dist(centre, box)^2 <= r^2 <= max dist^2, binary64
    const double h = (double)S / (double)(1 << D);
    const int res = 1 << D;
    for (int s = 0; s < ns; ++s) {
        const float* P = spheres + 4 * s;
        double ctr[3] = {P[0], P[1], P[2]};
        double r = P[3];
        double r2 = r * r;
        int lo_i[3], hi_i[3];
        for (int a = 0; a < 3; ++a) {
            lo_i[a] = std::max(0, (int)std::floor((ctr[a] - r - (double)lo[a]) / h) - 1);
            hi_i[a] = std::min(res - 1, (int)std::floor((ctr[a] + r - (double)lo[a]) / h) + 1);
        }
        for (int iz = lo_i[2]; iz <= hi_i[2]; ++iz)
            for (int iy = lo_i[1]; iy <= hi_i[1]; ++iy)
                for (int ix = lo_i[0]; ix <= hi_i[0]; ++ix) {
                    int idx[3] = {ix, iy, iz};
                    double dmin2 = 0, dmax2 = 0;
                    for (int a = 0; a < 3; ++a) {
                        double bl = (double)lo[a] + (double)idx[a] * h;
                        double bh = (double)lo[a] + (double)(idx[a] + 1) * h;
                        double e = std::max(0.0, std::max(bl - ctr[a], ctr[a] - bh));
                        dmin2 = dmin2 + e * e;
                        double m = std::max(std::fabs(ctr[a] - bl), std::fabs(ctr[a] - bh));
                        dmax2 = dmax2 + m * m;
                    }
                    if (dmin2 <= r2 && r2 <= dmax2)
                        out.push_back({morton((uint32_t)ix, (uint32_t)iy, (uint32_t)iz),
                                       (uint32_t)(nq + s)});
                }
    }
    // triangles: every voxel of the vertices' bounding box widened by one, by the SAT test
    for (int t = 0; t < nt; ++t) {
        const float* T = tris + 9 * t;
        int lo_i[3], hi_i[3];
        for (int a = 0; a < 3; ++a) {
            double mn = std::min((double)T[a], std::min((double)T[3 + a], (double)T[6 + a]));
            double mx = std::max((double)T[a], std::max((double)T[3 + a], (double)T[6 + a]));
            lo_i[a] = (int)std::max(0.0, std::floor((mn - (double)lo[a]) / h) - 1.0);
            hi_i[a] = (int)std::min((double)(res - 1), std::floor((mx - (double)lo[a]) / h) + 1.0);
        }
        for (int iz = lo_i[2]; iz <= hi_i[2]; ++iz)
            for (int iy = lo_i[1]; iy <= hi_i[1]; ++iy)
                for (int ix = lo_i[0]; ix <= hi_i[0]; ++ix) {
                    int idx[3] = {ix, iy, iz};
                    double c[3];
                    for (int a = 0; a < 3; ++a) c[a] = (double)lo[a] + ((double)idx[a] + 0.5) * h;
                    if (tri_box_overlap(T, c, h * 0.5))
                        out.push_back({morton((uint32_t)ix, (uint32_t)iy, (uint32_t)iz),
                                       (uint32_t)(nq + ns + t)});
                }
    }
}

// analytic normal of primitive `prim` for the fragment in leaf (ix, iy, iz):
// quads use their stored normal, spheres the direction from the centre to the
// voxel centre (the normal at the surface point nearest the voxel centre),
// triangles their geometric normal (v1 - v0) x (v2 - v0), normalised
void frag_normal(const float* quads, int nq, const float* spheres, int ns, const float* tris, const Svo& s,
                 uint32_t prim, uint64_t key, float out[3]) {
    if ((int)prim >= nq + ns) {
        const float* T = tris + 9 * (prim - nq - ns);
        float e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = T[3 + a] - T[a];
            e2[a] = T[6 + a] - T[a];
        }
        float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        float len2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        if (len2 > 0) {
            float len = std::sqrt(len2);
            out[0] = n[0] / len;
            out[1] = n[1] / len;
            out[2] = n[2] / len;
        } else {
            out[0] = 0.0f;
            out[1] = 1.0f;
            out[2] = 0.0f;
        }
        return;
    }
    if ((int)prim < nq) {
        const float* Q = quads + 8 * prim;
        int a = (int)Q[0];
        out[0] = out[1] = out[2] = 0.0f;
        out[a] = Q[6];
        return;
    }
    const float* P = spheres + 4 * (prim - nq);
    uint32_t c[3];
    morton_decode(key, &c[0], &c[1], &c[2]);
    const float h = s.S / (float)(1 << s.D);
    float dv[3];
    for (int a = 0; a < 3; ++a) {
        float vc = s.lo[a] + ((float)c[a] + 0.5f) * h;
        dv[a] = vc - P[a];
    }
    float len2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
    if (len2 > 0) {
        float len = std::sqrt(len2);
        out[0] = dv[0] / len;
        out[1] = dv[1] / len;
        out[2] = dv[2] / len;
    } else {
        out[0] = 0.0f;
        out[1] = 1.0f;
        out[2] = 0.0f;
    }
}

}  // namespace

Svo* build_svo(const float* quads, int nq, const float* spheres, int ns, const float* tris, int nt,
               const float lo[3], float S, int D) {
    std::vector<Frag> frags;
    voxelize(quads, nq, spheres, ns, tris, nt, lo, S, D, frags);
    if (frags.empty()) return nullptr;
    std::sort(frags.begin(), frags.end());

    Svo* s = new Svo();
    s->D = D;
    for (int a = 0; a < 3; ++a) s->lo[a] = lo[a];
    s->S = S;
    s->scale = (float)(1 << D) / S;
    s->keys.assign(D + 1, {});
    // leaves and their fragment lists
    for (size_t i = 0; i < frags.size(); ++i) {
        if (i == 0 || frags[i].key != frags[i - 1].key) {
            s->keys[D].push_back(frags[i].key);
            s->frag_off.push_back((uint32_t)i);
        }
        s->frag_prim.push_back(frags[i].prim);
    }
    s->frag_off.push_back((uint32_t)frags.size());
    // inner levels: unique prefixes
    for (int l = D - 1; l >= 0; --l) {
        for (uint64_t k : s->keys[l + 1]) {
            uint64_t p = k >> 3;
            if (s->keys[l].empty() || s->keys[l].back() != p) s->keys[l].push_back(p);
        }
    }
    s->level_off.assign(D + 2, 0);
    for (int l = 0; l <= D; ++l) s->level_off[l + 1] = s->level_off[l] + (uint32_t)s->keys[l].size();
    const uint32_t n = s->num_nodes();
    s->first_child.assign(n, NONE);
    s->parent.assign(n, NONE);
    s->child_mask.assign(n, 0);
    s->leaf_count.assign(n, 0);
    s->normal.assign(3 * (size_t)n, 0.0f);
    for (int l = 0; l < D; ++l) {
        const std::vector<uint64_t>& ck = s->keys[l + 1];
        for (size_t j = 0; j < ck.size(); ++j) {
            uint32_t child = s->level_off[l + 1] + (uint32_t)j;
            uint32_t par = s->find(l, ck[j] >> 3);
            s->parent[child] = par;
            if (s->first_child[par] == NONE) s->first_child[par] = child;
            s->child_mask[par] |= (uint8_t)(1u << (ck[j] & 7));
        }
    }
    // leaf normals from the fragments of each leaf
    std::vector<float> fn, fw;
    for (size_t j = 0; j < s->keys[D].size(); ++j) {
        uint32_t node = s->level_off[D] + (uint32_t)j;
        uint32_t b = s->frag_off[j], e = s->frag_off[j + 1];
        fn.assign(3 * (e - b), 0.0f);
        fw.assign(e - b, 1.0f);
        for (uint32_t f = b; f < e; ++f)
            frag_normal(quads, nq, spheres, ns, tris, *s, s->frag_prim[f], s->keys[D][j], &fn[3 * (f - b)]);
        kmeans2(fn.data(), fw.data(), (int)(e - b), &s->normal[3 * (size_t)node]);
        s->leaf_count[node] = 1;
    }
    // inner normals: k-means over the children's normals weighted by leaf count
    for (int l = D - 1; l >= 0; --l) {
        for (uint32_t node = s->level_off[l]; node < s->level_off[l + 1]; ++node) {
            int m = __builtin_popcount(s->child_mask[node]);
            fn.assign(3 * m, 0.0f);
            fw.assign(m, 0.0f);
            uint32_t cnt = 0;
            for (int c = 0; c < m; ++c) {
                uint32_t ch = s->first_child[node] + c;
                for (int a = 0; a < 3; ++a) fn[3 * c + a] = s->normal[3 * (size_t)ch + a];
                fw[c] = (float)s->leaf_count[ch];
                cnt += s->leaf_count[ch];
            }
            kmeans2(fn.data(), fw.data(), m, &s->normal[3 * (size_t)node]);
            s->leaf_count[node] = cnt;
        }
    }
    s->acc_sum.assign(2 * (size_t)n, 0);
    s->tot_sum.assign(2 * (size_t)n, 0);
    s->acc_cnt.assign(2 * (size_t)n, 0);
    s->tot_cnt.assign(2 * (size_t)n, 0);
    s->value.assign(2 * (size_t)n, 0.0f);
    return s;
}

// UpdateExitance (Alg. 1, Eq. 5): each record (position, outgoing direction,
// local radiance estimate L) is added to the deepest existing node holding its
// position, on the side whose normal faces the outgoing direction
// (dot(N, w_out) >= 0 -> side 0 (N), else side 1 (-N)).  Reading: the paper
// accumulates floats with atomics; here L is quantised to 2^-20 (clamped to
// [0, 2^24]) and summed as unsigned 64-bit integers, so the sum does not
// depend on the order of the records.
void accumulate(Svo& s, const float* pos, const float* wout, const float* L, size_t n) {
    for (size_t i = 0; i < n; ++i) {
        uint32_t node = s.deepest(pos + 3 * i);
        if (node == NONE) continue;
        const float* N = &s.normal[3 * (size_t)node];
        const float* w = wout + 3 * i;
        float d = N[0] * w[0] + N[1] * w[1] + N[2] * w[2];
        int side = (d >= 0.0f) ? 0 : 1;
        float Lc = (L[i] > 0.0f) ? std::min(L[i], 16777216.0f) : 0.0f;
        uint64_t q = (uint64_t)std::nearbyint(Lc * 1048576.0f);
        s.acc_sum[2 * (size_t)node + side] += q;
        s.acc_cnt[2 * (size_t)node + side] += 1;
    }
}

// Bottom-up averaging (Sec. 3.2).  Reading: the average is weighted by record
// count -- a node's integer sums are its own records plus its children's sums,
// each child side routed to the parent side its normal agrees with
// (dot(+-N_child, N_parent) >= 0 -> parent side 0).  The value of a side is
// sum * 2^-20 / count; an empty side takes the other side's value, else 0.
void reduce(Svo& s) {
    const int D = s.D;
    for (uint32_t node = s.level_off[D]; node < s.level_off[D + 1]; ++node) {
        for (int k = 0; k < 2; ++k) {
            s.tot_sum[2 * (size_t)node + k] = s.acc_sum[2 * (size_t)node + k];
            s.tot_cnt[2 * (size_t)node + k] = s.acc_cnt[2 * (size_t)node + k];
        }
    }
    for (int l = D - 1; l >= 0; --l) {
        for (uint32_t node = s.level_off[l]; node < s.level_off[l + 1]; ++node) {
            uint64_t sum[2] = {s.acc_sum[2 * (size_t)node], s.acc_sum[2 * (size_t)node + 1]};
            uint32_t cnt[2] = {s.acc_cnt[2 * (size_t)node], s.acc_cnt[2 * (size_t)node + 1]};
            const float* P = &s.normal[3 * (size_t)node];
            int m = __builtin_popcount(s.child_mask[node]);
            for (int c = 0; c < m; ++c) {
                uint32_t ch = s.first_child[node] + c;
                const float* C = &s.normal[3 * (size_t)ch];
                float dpos = C[0] * P[0] + C[1] * P[1] + C[2] * P[2];
                float nC[3] = {-C[0], -C[1], -C[2]};
                float dneg = nC[0] * P[0] + nC[1] * P[1] + nC[2] * P[2];
                int p0 = (dpos >= 0.0f) ? 0 : 1;
                int p1 = (dneg >= 0.0f) ? 0 : 1;
                sum[p0] += s.tot_sum[2 * (size_t)ch];
                cnt[p0] += s.tot_cnt[2 * (size_t)ch];
                sum[p1] += s.tot_sum[2 * (size_t)ch + 1];
                cnt[p1] += s.tot_cnt[2 * (size_t)ch + 1];
            }
            for (int k = 0; k < 2; ++k) {
                s.tot_sum[2 * (size_t)node + k] = sum[k];
                s.tot_cnt[2 * (size_t)node + k] = cnt[k];
            }
        }
    }
    const uint32_t n = s.num_nodes();
    for (uint32_t node = 0; node < n; ++node) {
        float v[2];
        bool has[2];
        for (int k = 0; k < 2; ++k) {
            uint32_t c = s.tot_cnt[2 * (size_t)node + k];
            has[k] = c != 0;
            v[k] = has[k] ? ((float)s.tot_sum[2 * (size_t)node + k] * 0x1p-20f) / (float)c : 0.0f;
        }
        for (int k = 0; k < 2; ++k) {
            if (!has[k]) v[k] = has[1 - k] ? v[1 - k] : 0.0f;
            s.value[2 * (size_t)node + k] = v[k];
        }
    }
}

}  // namespace orc
