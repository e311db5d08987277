/* CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain C entry points of the CPU oracle for the wavefront path-guiding hot
 * path.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  All pointers are host pointers owned by the caller;
 * handles returned by orc_svo_build are freed with orc_svo_free.
 *
 * Parity pins: every function here is checked by the CPU test suite against
 * facts that do not come from the oracle itself (brute force on tiny inputs,
 * closed forms, special cases, statistical tests).  The exact values of the
 * cone-traced radiance against the paper's own renderer are unpinned: the
 * paper's scenes and code are not available.
 */
#ifndef WFPG_ORACLE_H
#define WFPG_ORACLE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* SVO build (Sec. 3.2): conservative voxelisation, Morton sort, hierarchy,
 * k-means normals.  NULL if the scene occupies no voxel. */
void* orc_svo_build(const float* quads, int nq, const float* spheres, int ns, const float* tris, int nt,
                    const float* lo, float S, int D);
void orc_svo_free(void* svo);
uint32_t orc_svo_num_nodes(const void* svo);
void orc_svo_level_off(const void* svo, uint32_t* out /* D + 2 */);
/* per node in global-id order: Morton prefix at its level, first child (global
 * id, 0xFFFFFFFF for leaves), child mask, parent, normal (3 floats), leaf count */
void orc_svo_export(const void* svo, uint64_t* key, uint32_t* first_child, uint8_t* mask,
                    uint32_t* parent, float* normal, uint32_t* leaf_count);
/* fragment lists of the leaves: offsets (leaves + 1) and primitive ids */
uint32_t orc_svo_num_frags(const void* svo);
void orc_svo_export_frags(const void* svo, uint32_t* off, uint32_t* prim);
uint32_t orc_svo_deepest(const void* svo, const float* p);

/* UpdateExitance (Eq. 5, Alg. 1) then the bottom-up average */
void orc_svo_accumulate(void* svo, const float* pos, const float* wout, const float* L, size_t n);
void orc_svo_export_exitance(const void* svo, uint64_t* acc_sum, uint32_t* acc_cnt,
                             uint64_t* tot_sum, uint32_t* tot_cnt, float* value);

/* Partition-S (Alg. 2, mode 0) or runs of given sizes (mode 1), then the
 * choice of origins.  Returns the bin count; -1 on bad sizes; -2 if the bin
 * count exceeds bin_cap (nothing written). */
int64_t orc_bin_rays(const void* svo, const float* pos, const float* nrm, size_t n, int mode,
                     int l_min, uint32_t c_ray, const uint32_t* sizes, uint32_t n_sizes,
                     uint64_t seed, uint32_t frame, uint32_t* bin_of_ray, uint32_t* ray_order,
                     uint32_t* bin_offset, uint32_t* origin_ray, uint32_t bin_cap);

/* GuideRays field + PDF/CDF (Alg. 3) for nb bins with the given origins; bin
 * ids select the jitter streams.  field receives the blurred field.  steps
 * (if not NULL) accumulates the leaf cells the cone rays entered; blocks (if
 * not NULL) the maximal empty blocks and leaves they passed (slow). */
void orc_guide_build(const void* svo, const float* origins, const uint32_t* bin_ids, uint32_t nb,
                     int N, float eps, int jitter, int blur, float t_skip, int cos_weight,
                     uint64_t seed, uint32_t frame, float* field, float* pdf, float* cdf_row,
                     float* cdf_marg, uint64_t* steps, uint64_t* blocks);
void orc_guide_sample(const float* pdf, const float* cdf_row, const float* cdf_marg, int N,
                      const uint32_t* bin, const float* u, size_t n, float* dir, float* p,
                      uint32_t* cell);
void orc_guide_eval_pdf(const float* pdf, int N, const uint32_t* bin, const float* dir, size_t n,
                        float* out);

/* building blocks, exposed for the pins */
uint64_t orc_morton(uint32_t x, uint32_t y, uint32_t z);
uint64_t orc_rng_u64(uint64_t seed, uint64_t stream, uint64_t counter);
float orc_sin(float x);
float orc_cos(float x);
float orc_atan01(float q);
void orc_octa_decode(const float* uv, size_t n, float* out);
void orc_octa_encode(const float* d, size_t n, float* out);
void orc_kmeans2(const float* n, const float* w, int m, float* out);
void orc_warp_scan(float* x, int n);
void orc_blur(float* f, int N);
void orc_pdf_cdf(const float* f, int N, float* pdf, float* cdf_row, float* cdf_marg);
void orc_trace(const void* svo, const float* o, const float* d, size_t n, float t_skip,
               float omega, int cos_weight, int32_t* hit, uint64_t* leaf_key, float* t_entry,
               int32_t* level, uint32_t* node, int32_t* side, float* value, uint32_t* steps,
               uint32_t* blocks);

#ifdef __cplusplus
}
#endif
#endif
