// CPU ORACLE -- TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
// extern "C" entry points declared in oracle.h.
#include <cstring>
#include <vector>

#include "oracle.h"
#include "oracle_internal.h"

namespace orc {
void accumulate(Svo& s, const float* pos, const float* wout, const float* L, size_t n);
void reduce(Svo& s);
uint32_t partition_s(const Svo& s, const float* pos, size_t n, int l_min, uint32_t c_ray,
                     uint32_t* bin_of_ray, uint32_t* ray_order, std::vector<uint32_t>& bin_offset);
uint32_t partition_runs(const Svo& s, const float* pos, const float* nrm, size_t n,
                        const uint32_t* sizes, uint32_t nb, uint32_t* bin_of_ray,
                        uint32_t* ray_order, std::vector<uint32_t>& bin_offset);
void select_origins(const uint32_t* ray_order, const std::vector<uint32_t>& bin_offset,
                    uint32_t nb, uint64_t seed, uint32_t frame, uint32_t* origin_ray);
void build_field(const Svo& s, const float o[3], uint32_t bin, int N, float eps, int jitter,
                 float t_skip, int cos_weight, uint64_t seed, uint32_t frame, float* f,
                 uint64_t* steps, uint64_t* blocks);
void blur_field(float* f, int N);
void warp_order_scan(float* x, int n);
void pdf_cdf(const float* f, int N, float* pdf, float* cdf_row, float* cdf_marg);
void sample_one(const float* pdf, const float* cdf_row, const float* cdf_marg, int N, float u0,
                float u1, float dir[3], float* p, uint32_t* cell);
float eval_one(const float* pdf, int N, const float d[3]);
}  // namespace orc

using namespace orc;

extern "C" {

void* orc_svo_build(const float* quads, int nq, const float* spheres, int ns, const float* tris, int nt,
                    const float* lo, float S, int D) {
    return build_svo(quads, nq, spheres, ns, tris, nt, lo, S, D);
}
void orc_svo_free(void* s) { delete static_cast<Svo*>(s); }
uint32_t orc_svo_num_nodes(const void* s) { return static_cast<const Svo*>(s)->num_nodes(); }
void orc_svo_level_off(const void* sv, uint32_t* out) {
    const Svo* s = static_cast<const Svo*>(sv);
    for (int l = 0; l <= s->D + 1; ++l) out[l] = s->level_off[l];
}
void orc_svo_export(const void* sv, uint64_t* key, uint32_t* first_child, uint8_t* mask,
                    uint32_t* parent, float* normal, uint32_t* leaf_count) {
    const Svo* s = static_cast<const Svo*>(sv);
    const uint32_t n = s->num_nodes();
    for (int l = 0; l <= s->D; ++l)
        for (size_t j = 0; j < s->keys[l].size(); ++j) key[s->level_off[l] + j] = s->keys[l][j];
    std::memcpy(first_child, s->first_child.data(), n * 4);
    std::memcpy(mask, s->child_mask.data(), n);
    std::memcpy(parent, s->parent.data(), n * 4);
    std::memcpy(normal, s->normal.data(), (size_t)n * 12);
    std::memcpy(leaf_count, s->leaf_count.data(), n * 4);
}
uint32_t orc_svo_num_frags(const void* sv) {
    return (uint32_t)static_cast<const Svo*>(sv)->frag_prim.size();
}
void orc_svo_export_frags(const void* sv, uint32_t* off, uint32_t* prim) {
    const Svo* s = static_cast<const Svo*>(sv);
    std::memcpy(off, s->frag_off.data(), s->frag_off.size() * 4);
    std::memcpy(prim, s->frag_prim.data(), s->frag_prim.size() * 4);
}
uint32_t orc_svo_deepest(const void* s, const float* p) {
    return static_cast<const Svo*>(s)->deepest(p);
}

void orc_svo_accumulate(void* sv, const float* pos, const float* wout, const float* L, size_t n) {
    Svo* s = static_cast<Svo*>(sv);
    accumulate(*s, pos, wout, L, n);
    reduce(*s);
}
void orc_svo_export_exitance(const void* sv, uint64_t* acc_sum, uint32_t* acc_cnt,
                             uint64_t* tot_sum, uint32_t* tot_cnt, float* value) {
    const Svo* s = static_cast<const Svo*>(sv);
    const size_t n = 2 * (size_t)s->num_nodes();
    std::memcpy(acc_sum, s->acc_sum.data(), n * 8);
    std::memcpy(acc_cnt, s->acc_cnt.data(), n * 4);
    std::memcpy(tot_sum, s->tot_sum.data(), n * 8);
    std::memcpy(tot_cnt, s->tot_cnt.data(), n * 4);
    std::memcpy(value, s->value.data(), n * 4);
}

int64_t orc_bin_rays(const void* sv, const float* pos, const float* nrm, size_t n, int mode,
                     int l_min, uint32_t c_ray, const uint32_t* sizes, uint32_t n_sizes,
                     uint64_t seed, uint32_t frame, uint32_t* bin_of_ray, uint32_t* ray_order,
                     uint32_t* bin_offset, uint32_t* origin_ray, uint32_t bin_cap) {
    const Svo* s = static_cast<const Svo*>(sv);
    std::vector<uint32_t> b(n), o(n), off;
    uint32_t nb;
    if (mode == 0) {
        nb = partition_s(*s, pos, n, l_min, c_ray, b.data(), o.data(), off);
    } else {
        nb = partition_runs(*s, pos, nrm, n, sizes, n_sizes, b.data(), o.data(), off);
        if (nb == 0) return -1;
    }
    if (nb > bin_cap) return -2;
    std::memcpy(bin_of_ray, b.data(), n * 4);
    std::memcpy(ray_order, o.data(), n * 4);
    std::memcpy(bin_offset, off.data(), (nb + 1) * 4);
    select_origins(o.data(), off, nb, seed, frame, origin_ray);
    return nb;
}

void orc_guide_build(const void* sv, const float* origins, const uint32_t* bin_ids, uint32_t nb,
                     int N, float eps, int jitter, int blur, float t_skip, int cos_weight,
                     uint64_t seed, uint32_t frame, float* field, float* pdf, float* cdf_row,
                     float* cdf_marg, uint64_t* steps, uint64_t* blocks) {
    const Svo* s = static_cast<const Svo*>(sv);
    const size_t NN = (size_t)N * N;
    for (uint32_t k = 0; k < nb; ++k) {
        float* f = field + k * NN;
        build_field(*s, origins + 3 * k, bin_ids[k], N, eps, jitter, t_skip, cos_weight, seed,
                    frame, f, steps, blocks);
        if (blur) blur_field(f, N);
        pdf_cdf(f, N, pdf + k * NN, cdf_row + k * NN, cdf_marg + (size_t)k * N);
    }
}

void orc_guide_sample(const float* pdf, const float* cdf_row, const float* cdf_marg, int N,
                      const uint32_t* bin, const float* u, size_t n, float* dir, float* p,
                      uint32_t* cell) {
    const size_t NN = (size_t)N * N;
    for (size_t i = 0; i < n; ++i) {
        size_t b = bin[i];
        sample_one(pdf + b * NN, cdf_row + b * NN, cdf_marg + b * N, N, u[2 * i], u[2 * i + 1],
                   dir + 3 * i, p + i, cell + i);
    }
}

void orc_guide_eval_pdf(const float* pdf, int N, const uint32_t* bin, const float* dir, size_t n,
                        float* out) {
    const size_t NN = (size_t)N * N;
    for (size_t i = 0; i < n; ++i) out[i] = eval_one(pdf + bin[i] * NN, N, dir + 3 * i);
}

uint64_t orc_morton(uint32_t x, uint32_t y, uint32_t z) { return morton(x, y, z); }
uint64_t orc_rng_u64(uint64_t seed, uint64_t stream, uint64_t counter) {
    return rng_u64(seed, stream, counter);
}
float orc_sin(float x) { return poly_sin(x); }
float orc_cos(float x) { return poly_cos(x); }
float orc_atan01(float q) { return poly_atan01(q); }
void orc_octa_decode(const float* uv, size_t n, float* out) {
    for (size_t i = 0; i < n; ++i) octa_decode(uv[2 * i], uv[2 * i + 1], out + 3 * i);
}
void orc_octa_encode(const float* d, size_t n, float* out) {
    for (size_t i = 0; i < n; ++i) octa_encode(d + 3 * i, out + 2 * i, out + 2 * i + 1);
}
void orc_kmeans2(const float* n, const float* w, int m, float* out) { kmeans2(n, w, m, out); }
void orc_warp_scan(float* x, int n) { warp_order_scan(x, n); }
void orc_blur(float* f, int N) { blur_field(f, N); }
void orc_pdf_cdf(const float* f, int N, float* pdf, float* cdf_row, float* cdf_marg) {
    pdf_cdf(f, N, pdf, cdf_row, cdf_marg);
}
void orc_trace(const void* sv, const float* o, const float* d, size_t n, float t_skip,
               float omega, int cos_weight, int32_t* hit, uint64_t* leaf_key, float* t_entry,
               int32_t* level, uint32_t* node, int32_t* side, float* value, uint32_t* steps,
               uint32_t* blocks) {
    const Svo* s = static_cast<const Svo*>(sv);
    for (size_t i = 0; i < n; ++i) {
        TraceResult r = trace_cell(*s, o + 3 * i, d + 3 * i, t_skip, omega, cos_weight, blocks != nullptr);
        if (blocks) blocks[i] = r.blocks;
        hit[i] = r.hit;
        leaf_key[i] = r.hit ? r.leaf_key : 0;
        t_entry[i] = r.hit ? r.t_entry : 0.0f;
        level[i] = r.hit ? r.level : -1;
        node[i] = r.node;
        side[i] = r.hit ? r.side : -1;
        value[i] = r.value;
        steps[i] = r.steps;
    }
}

}  // extern "C"
