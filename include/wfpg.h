/*
 * wfpg.h -- C ABI of the GB300 (sm_103a) wavefront path-guiding hot path.
 *
 * Method: Yalciner & Akyuz, "Path Guiding for Wavefront Path Tracing: A
 * Memory Efficient Approach for GPU Path Tracers".  Radiant exitance from
 * path vertices is cached in one sparse voxel octree (SVO, Sec. 3.2); rays
 * are binned by position with the SVO (Sec. 3.4, Alg. 2); for each bin a
 * directional radiance field is cone-traced through the SVO from one origin
 * (Sec. 3.3, Eq. 6, Alg. 3) and turned into a piecewise-constant PDF/CDF on
 * the concentric octahedral map (Sec. 3.5, Sec. 3 "Implementation"), which
 * every ray of the bin samples and which MIS evaluates.
 *
 * Conventions shared by every entry point:
 *  - Return value: WFPG_OK (0) or a negative WFPG_ERR_* code; the message of
 *    the last failure on the calling thread is wfpg_last_error().  Nothing is
 *    thrown across the ABI and the library never exits the process.
 *  - Array arguments are DEVICE pointers owned by the caller (for instance
 *    torch tensors' data_ptr()), unless a comment says "host".  Layouts are
 *    stated per argument; "xyz" arrays are n x 3 float32, row-major.
 *  - `stream` is a cudaStream_t passed as void*.  Work is enqueued on it and
 *    the call returns without synchronising, except where a comment says the
 *    call synchronises (svo_build, the export calls, wfpg_svo_status).
 *  - The SVO handle is owned by the library: svo_build creates it,
 *    svo_destroy frees it.  Device-side problems (an iteration cap reached, a
 *    bin count above the caller's capacity, run sizes that do not add up) set
 *    bits of the handle's status word; wfpg_svo_status reads them.
 *  - Levels are numbered from the root = 0 to the leaves = depth (the paper
 *    counts the root as level 1: its l_min = k is l_min = k - 1 here).
 */
#ifndef WFPG_H
#define WFPG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define WFPG_API __attribute__((visibility("default")))
#else
#define WFPG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    WFPG_OK = 0,
    WFPG_ERR_INVALID_ARG = -1,
    WFPG_ERR_OOM = -2,
    WFPG_ERR_CUDA = -3,
    WFPG_ERR_TIMEOUT = -4,
    WFPG_ERR_CAPACITY = -5
};

/* bits of the device status word */
enum {
    WFPG_STATUS_TRACE_CAP = 1u << 0,    /* a cone ray hit the walk's step cap (treated as a miss) */
    WFPG_STATUS_BIN_CAPACITY = 1u << 1, /* bin_rays found more bins than bin_cap */
    WFPG_STATUS_RUN_SIZES = 1u << 2,    /* run sizes do not add up to the ray count */
    WFPG_STATUS_MMA_TIMEOUT = 1u << 3,  /* a tensor-core wait hit its limit (results invalid) */
    WFPG_STATUS_WAIT_TIMEOUT = 1u << 4  /* a block's wait for an earlier block of the same launch
                                           hit its limit (the sort behind bin_rays; results invalid) */
};

#define WFPG_MAX_DEPTH 11

/* Scene, device arrays owned by the caller.
 *  quads   n_quads x 8 float32: axis, plane, lo1, hi1, lo2, hi2, nsign, 0 --
 *          the quad lies in x[axis] = plane, spans [lo1, hi1] on axis
 *          (axis+1)%3 and [lo2, hi2] on axis (axis+2)%3, normal nsign*e_axis.
 *  spheres n_spheres x 4 float32: cx, cy, cz, r.
 *  tris    n_tris x 9 float32: v0, v1, v2 (triangle meshes, Sec. 3.2); the
 *          fragment normal is the winding normal (v1 - v0) x (v2 - v0).
 *  Primitive ids count the quads, then the spheres, then the triangles
 *  (at most 2^20 primitives in all).
 *  lo, size: host values, the cubic AABB [lo, lo + size]^3 voxelised. */
typedef struct wfpg_scene {
    const float* quads;
    uint32_t n_quads;
    const float* spheres;
    uint32_t n_spheres;
    float lo[3];
    float size;
    const float* tris;
    uint32_t n_tris;
} wfpg_scene;

typedef struct wfpg_svo wfpg_svo;

/* Read-only description of a built SVO; the device pointers stay valid until
 * svo_destroy.  Node arrays are indexed by global node id = level_off[l] +
 * index within level l (levels hold Morton-sorted unique prefixes). */
typedef struct wfpg_svo_info {
    int depth;
    uint32_t n_nodes;
    uint32_t n_frags;
    uint32_t level_off[WFPG_MAX_DEPTH + 2];
    const void* node;          /* n_nodes x {uint32 first_child, uint32 child_mask} */
    const uint32_t* parent;    /* n_nodes, 0xFFFFFFFF for the root */
    const float* normal;       /* n_nodes x 4 (nx, ny, nz, 0): side 0 is N, side 1 is -N */
    const float* value;        /* n_nodes x 2 averaged exitance per side */
} wfpg_svo_info;

/*
 * svo_build -- SVO generation (Sec. 3.2; Table 1 "SVO generation").
 * Conservative voxelisation of the scene at 2^depth leaves per axis (a voxel
 * is occupied when a primitive's surface meets the closed voxel box; the
 * paper rasterises triangles after Crassin & Green), Morton-key radix sort,
 * level-by-level node allocation, and two normals per node from k-means with
 * k = 2 (Fig. 2).  depth in [1, WFPG_MAX_DEPTH].  Synchronises `stream`.
 * Besides the tree it builds the walk's index: a dense grid per level 0 ..
 * min(6, depth) holding each cell's deepest existing node, and for depths up
 * to 11 an occupancy bitmap per deeper level (8^l bits for level l: 18 MB at
 * depth 9, 1.2 GB at depth 11), with which guide_build_pdf marches every bin's
 * cone rays as one stream.
 * Errors: INVALID_ARG (depth, counts, empty scene), OOM, CUDA.
 */
WFPG_API int svo_build(const wfpg_scene* scene, int depth, void* stream, wfpg_svo** out);
WFPG_API int svo_destroy(wfpg_svo* svo);
WFPG_API int svo_get_info(const wfpg_svo* svo, wfpg_svo_info* out /* host */);

/*
 * svo_reset_exitance -- zero the accumulated records (all sums and counts).
 */
WFPG_API int svo_reset_exitance(wfpg_svo* svo, void* stream);

/*
 * svo_accumulate -- UpdateExitance (Alg. 1; Eq. 5) followed by the
 * bottom-up average (Sec. 3.2).  n records: pos (xyz), wout (xyz, the
 * direction the radiance leaves toward, unit) and L (float32, the local
 * radiance estimate of Eq. 5).  Each record adds round(clamp(L, 0, 2^24) *
 * 2^20) to the unsigned 64-bit sum, and 1 to the count, of the deepest
 * existing node holding pos, on side 0 if dot(N, wout) >= 0 else side 1.
 * Sums persist across calls (a running mean).  Then every inner node's sums
 * are recomputed from its own records and its children's sums (each child
 * side routed to the parent side its normal agrees with) and every node's
 * value[s] = sum * 2^-20 / count (an empty side takes the other side's value,
 * else 0).  n may be 0 (only the average is recomputed).
 */
WFPG_API int svo_accumulate(wfpg_svo* svo, const float* pos, const float* wout, const float* L,
                   uint32_t n, void* stream);

/* Binning modes */
enum {
    WFPG_BIN_PARTITION_S = 0, /* Alg. 2 */
    WFPG_BIN_RUNS = 1         /* stand-in for bins of a given length mix, see bin_rays */
};

typedef struct wfpg_bin_params {
    int mode;          /* WFPG_BIN_PARTITION_S or WFPG_BIN_RUNS */
    int l_min;         /* PARTITION_S: lowest level a bin may be (root = 0), clamped to [0, depth] */
    uint32_t c_ray;    /* PARTITION_S: ray-count threshold (0xFFFFFFFF: bins at l_min) */
    uint32_t n_sizes;  /* RUNS: number of runs (= bins) */
    uint64_t seed;     /* SelectOrigin random stream */
    uint32_t frame;    /* SelectOrigin random stream */
    const uint32_t* n_dev; /* optional DEVICE count of valid rays (the first *n_dev of the n); NULL: all n */
} wfpg_bin_params;

/*
 * bin_rays_workspace_size -- bytes of device scratch bin_rays needs for n rays
 * (host call, no device work).
 */
WFPG_API int bin_rays_workspace_size(const wfpg_svo* svo, uint32_t n, const wfpg_bin_params* p,
                            size_t* bytes /* host */);

/*
 * bin_rays -- Partition-S (Alg. 2; Sec. 3.4) and SelectOrigin (Sec. 3
 * "Implementation").
 * PARTITION_S: every ray descends to the deepest existing node holding pos
 * and counts there; for levels depth .. l_min a node's total is its own
 * count plus its children's totals and it is marked when total >= c_ray or
 * at l_min; each ray ascends to its first marked node (itself included; a
 * ray whose node lies above l_min keeps its node); bins are numbered by
 * ascending node id.
 * RUNS: rays are keyed by their cell at level min(6, depth) (Morton order)
 * and the octant of nrm, stably sorted by key, and the sorted sequence is cut
 * into runs of the given `sizes` (device, n_sizes uint32, all > 0, summing to
 * n); run j is bin j.
 * Outputs (device, caller-owned): bin_of_ray[n]; ray_order[n] = rays stably
 * sorted by bin; bin_offset[bin_cap + 1] = exclusive prefix of bin sizes;
 * origin_ray[bin_cap] = for bin b the ray at position floor(u * size_b) of
 * its run, u the 24-bit uniform of (seed, frame, b); *n_bins_dev = bin count.
 * If the bin count exceeds bin_cap, bins >= bin_cap are not written and
 * WFPG_STATUS_BIN_CAPACITY is set.  `workspace` holds at least
 * bin_rays_workspace_size() bytes (256-byte aligned); its contents on entry
 * do not matter.  nrm (xyz) is only read in RUNS mode (may be NULL
 * otherwise), sizes only in RUNS mode.  The rays are ordered by a stable
 * radix sort whose blocks wait for earlier blocks' digit counts; each wait is
 * bounded, and WFPG_STATUS_WAIT_TIMEOUT is set (the bins are then invalid) if
 * one runs out.
 */
WFPG_API int bin_rays(const wfpg_svo* svo, const float* pos, const float* nrm, uint32_t n,
             const wfpg_bin_params* p, const uint32_t* sizes, uint32_t* bin_of_ray,
             uint32_t* ray_order, uint32_t* bin_offset, uint32_t* origin_ray, uint32_t bin_cap,
             uint32_t* n_bins_dev, void* workspace, size_t workspace_bytes, void* stream);

/* Size of the fixed device scratch used by bin_rays_static (32 MiB). */
#define WFPG_BIN_STATIC_SCRATCH_BYTES (32u << 20)

/*
 * bin_rays_static -- bin_rays for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface convenience of this
 * library.  Hosts that own all device memory through their own pool (an
 * engine with a fixed, pre-reserved budget) or that have no device allocator
 * to carve a workspace from (a plain C caller) cannot provide bin_rays'
 * workspace; this variant takes the same arguments minus the workspace and
 * uses instead one file-scope device array of WFPG_BIN_STATIC_SCRATCH_BYTES,
 * reserved on every GPU that loads the library and held until the process
 * exits.  It calls no cudaMalloc, cudaFree or allocating routine.
 * Limit: the scratch bin_rays_workspace_size() reports for the same call must
 * fit in WFPG_BIN_STATIC_SCRATCH_BYTES (about 2.7M rays in RUNS mode; in
 * PARTITION_S mode 4 more bytes per ray and 12 per SVO node count too), otherwise the call
 * returns WFPG_ERR_CAPACITY and does nothing.
 * The first call on each device looks up the array's device address with the
 * device current (make that first call before any stream capture); later
 * calls reuse it.  Every call on a device shares the one array and leaves its
 * contents behind; the call clears what must start at zero itself.  Calls
 * whose work overlaps on the GPU (in flight on two streams, or from two
 * threads, at once) race on the scratch and corrupt each other's results:
 * serialise them.
 */
WFPG_API int bin_rays_static(const wfpg_svo* svo, const float* pos, const float* nrm, uint32_t n,
                             const wfpg_bin_params* p, const uint32_t* sizes, uint32_t* bin_of_ray,
                             uint32_t* ray_order, uint32_t* bin_offset, uint32_t* origin_ray,
                             uint32_t bin_cap, uint32_t* n_bins_dev, void* stream);

typedef struct wfpg_guide_params {
    int N;             /* field side: 8, 16, 32, 64 or 128 (N x N cells) */
    float eps;         /* initial field value (the paper's epsilon = 1e-2) */
    int jitter;        /* 1: jittered direction per cell, 0: cell centre */
    int blur;          /* 1: separable [1 2 1]/4 blur with the octahedral mirror */
    float t_skip;      /* a hit leaf must be entered at t >= t_skip (world units) */
    int cos_weight;    /* 1: multiply the node value by |dot(N, d)| */
    uint64_t seed;     /* jitter random stream */
    uint32_t frame;    /* jitter random stream */
    int block;         /* tuning: threads that work on one bin (64, 128, 256; 0 = default) */
    int stage;         /* tuning: 1 stage cone directions in shared memory, -1 do not, 0 = default */
    uint32_t split;    /* guide_build_sample: bins with more rays than this are sampled by a second,
                          GPU-wide launch (0 = default 2048, 0xFFFFFFFF = never); results do not change */
    uint32_t parts;    /* guide_build_pdf: the cells of a bin are traced by this many CTAs (1, 2, 4 or 8),
                          the last one finishing the bin; 0 = auto: split while the parts of all bins
                          fit in one wave of resident CTAs (few bins); results do not change */
} wfpg_guide_params;

/*
 * guide_build_pdf -- GuideRays up to GeneratePDF-CDF (Alg. 3; Sec. 3.3 and
 * 3.5).  For each bin b < min(*n_bins_dev, bin_cap) (all bin_cap bins when
 * n_bins_dev is NULL): the origin is pos[origin_ray[b]] (pos[b] when
 * origin_ray is NULL); cell (i, j) (column i along u, row j along v) looks
 * along the octahedral image of its centre (or a jittered point, stream
 * (seed, frame, b)); the ray marches the SVO to the first occupied leaf
 * entered at t >= t_skip, takes the ancestor whose squared side is closest
 * to t^2 * 4 pi / N^2 (Eq. 6) and reads that node's value on the side facing
 * back along the ray; field = eps + value (0 on a miss), optionally blurred;
 * row CDFs and the marginal CDF are inclusive scans in warp order; pdf =
 * field / total * N^2 / (4 pi).
 * Outputs (device, caller-owned, float32): pdf[bin_cap][N*N],
 * cdf_row[bin_cap][N*N], cdf_marg[bin_cap][N].  Bins past the count are not
 * written.  The SVO holds the field kernel's bin counter (zeroed on the stream
 * before each launch): field calls on one SVO (this, guide_build_sample,
 * frames) must be ordered on the GPU, as its status word already requires.
 */
WFPG_API int guide_build_pdf(const wfpg_svo* svo, const float* pos, const uint32_t* origin_ray,
                    const uint32_t* n_bins_dev, uint32_t bin_cap, const wfpg_guide_params* p,
                    float* pdf, float* cdf_row, float* cdf_marg, void* stream);

/*
 * guide_build_sample -- GuideRays as Alg. 3 states it: the field, its PDF
 * and CDFs live in shared memory only, and the bin's own rays sample from them
 * (guided density or BSDF, MIS) before the CTA moves on; nothing per bin is
 * written to global memory.  One persistent launch over all bins.
 * After bin b's CDF is built, every ray r of the bin (ray_order[bin_offset[b]
 * .. bin_offset[b+1]), as bin_rays writes them) takes u[r] = (u0, u1, u2):
 * if u2 < alpha it samples the field exactly as guide_sample does with
 * (u0, u1), else a cosine-distributed direction about the unit normal nrm[r]
 * (Malley's method on the orthonormal frame of Duff et al. 2017).  dir[r]
 * (xyz) gets the direction, pdf_out[r] the one-sample mixture density
 * alpha * field density + (1 - alpha) * max(0, cos) / pi there (the field
 * density of a cosine sample is its cell's, as guide_eval_pdf gives).
 * pos, nrm, u: device, [n][3]; bins as bin_rays writes them; alpha in [0, 1].
 * A bin with more than p->split rays (a Zipf head bin can hold a large share
 * of the frame) copies its field and CDFs to a workspace slot and its rays are
 * drawn by a second launch over the whole GPU with the same arithmetic.
 * Rays of bins >= min(*n_bins_dev, bin_cap) are not written.  Errors: invalid
 * N / eps / alpha / block, or a null array, give WFPG_ERR_INVALID_ARG; a
 * workspace smaller than guide_build_sample_workspace_size gives
 * WFPG_ERR_CAPACITY.
 */
WFPG_API int guide_build_sample(const wfpg_svo* svo, const float* pos, const float* nrm,
                                const uint32_t* origin_ray, const uint32_t* n_bins_dev, uint32_t bin_cap,
                                const uint32_t* ray_order, const uint32_t* bin_offset, const float* u,
                                uint32_t n, float alpha, const wfpg_guide_params* p, float* dir, float* pdf_out,
                                void* workspace, size_t ws_bytes, void* stream);
/* Device workspace guide_build_sample needs for n rays (spill slots of the
 * bins larger than p->split: their fields and CDFs). */
WFPG_API int guide_build_sample_workspace_size(int N, uint32_t n, uint32_t split, size_t* bytes);

/*
 * guide_sample_mix -- the sampling step of guide_build_sample from stored
 * tables (as guide_build_pdf or guide_learned_build_pdf write them): ray i of
 * bin b = bin_of_ray[i] takes u[i] = (u0, u1, u2); if u2 < alpha the guided
 * inverse-CDF sample (as guide_sample), else the cosine direction about
 * nrm[i]; pdf_out[i] = alpha * pdf[b][cell(dir)] + (1 - alpha) * max(0, cos)
 * / pi.  A ray whose bin is >= min(*n_bins_dev, bin_cap) (NULL: bin_cap) has
 * no table and takes the cosine branch with density cos / pi.  Rays
 * i >= min(*n_dev, n) (NULL: n) are not written.  With the same field, the
 * results equal guide_build_sample's bit for bit.
 */
WFPG_API int guide_sample_mix(const float* pdf, const float* cdf_row, const float* cdf_marg, int N,
                              uint32_t bin_cap, const uint32_t* n_bins_dev, const uint32_t* bin_of_ray,
                              const float* nrm, const float* u, uint32_t n, const uint32_t* n_dev, float alpha,
                              float* dir, float* pdf_out, void* stream);

/*
 * Product path guiding (Sec. 3.6): the bin's field at 8 x 8 blocks of
 * b x b cells (b = N / 8; N = 8 .. 128) times the ray's Lambertian BSDF at the
 * same resolution, sampled in two stages -- a block, then a cell and a point in
 * it from the full-resolution field inside the block.  Definitions:
 *   S_B    = sum of the cell densities pdf_c of block B (row-major blocks,
 *            cells summed row by row);
 *   beta_B = max(0, n . w_B) + 2^-10, w_B the octahedral image of the block's
 *            centre (the floor keeps the density positive wherever the field is);
 *   Z      = running sum of beta_B S_B over B = 0 .. 63;
 *   p(w)   = beta_B pdf_c N^2 / (4 pi Z)   (normalised over the sphere).
 * Sampling with (u0, u1): block = first B whose running sum exceeds u0 Z; the
 * remainder picks the row inside the block by the running sum of its row sums,
 * u1 the cell of that row by the running sum of its cells, and the in-cell
 * offsets invert those sums linearly (as guide_sample does).  All sums run
 * sequentially in the stated order, binary32.
 *
 * guide_product_sums: S[bin][64] for bins < min(*n_bins_dev, bin_cap), from
 *   pdf tables as guide_build_pdf or guide_learned_build_pdf write them.
 * guide_product_sample: per ray i < min(*n_dev, n): u[i] = (u0, u1, u2); if
 *   u2 < alpha the product sample, else a cosine direction about nrm[i];
 *   pdf_out[i] = alpha * p(dir) + (1 - alpha) * max(0, cos) / pi; cell[i] (may
 *   be NULL) = the product-sampled cell, 0xFFFFFFFF for the cosine branch.  A
 *   ray whose bin has no table takes the cosine branch with alpha = 0.
 * guide_product_eval: the same mixture density of given directions.
 */
WFPG_API int guide_product_sums(const float* pdf, int N, uint32_t bin_cap, const uint32_t* n_bins_dev, float* S,
                                void* stream);
WFPG_API int guide_product_sample(const float* pdf, const float* S, int N, uint32_t bin_cap,
                                  const uint32_t* n_bins_dev, const uint32_t* bin_of_ray, const float* nrm,
                                  const float* u, uint32_t n, const uint32_t* n_dev, float alpha, float* dir,
                                  float* pdf_out, uint32_t* cell, void* stream);
WFPG_API int guide_product_eval(const float* pdf, const float* S, int N, uint32_t bin_cap,
                                const uint32_t* n_bins_dev, const uint32_t* bin, const float* nrm,
                                const float* dir, uint32_t n, float alpha, float* out, void* stream);

/*
 * guide_sample -- the guided branch of Alg. 3's sampling step: inverse-CDF
 * sampling of the piecewise-constant density.  Per ray: t0 = u0 * T; the row
 * is the first marginal entry > t0 (N-1 if none); t1 = u1 * T_row; the
 * column the first row-CDF entry > t1; the point inside the cell inverts the
 * CDF linearly; the direction is its octahedral image.
 * In: pdf/cdf_row/cdf_marg as written by guide_build_pdf for bin_cap bins of
 * side N; bin_of_ray[n]; u[n][2] in [0, 1).  Out: dir (xyz), pdf_out[n] (the
 * cell's density), cell[n] = row * N + column.  A ray whose bin is >= bin_cap
 * gets dir = 0, pdf 0, cell 0xFFFFFFFF.
 */
WFPG_API int guide_sample(const float* pdf, const float* cdf_row, const float* cdf_marg, int N,
                 uint32_t bin_cap, const uint32_t* bin_of_ray, const float* u, uint32_t n,
                 float* dir, float* pdf_out, uint32_t* cell, void* stream);

/*
 * guide_eval_pdf -- density of arbitrary directions (needed by MIS; Sec. 3
 * "Implementation"): the cell of dir under the octahedral map, i =
 * floor((u + 1) N / 2) clamped to [0, N-1] (same for the row), and that
 * cell's pdf.  bin[n], dir (xyz, unit) -> out[n]; bins >= bin_cap give 0.
 */
WFPG_API int guide_eval_pdf(const float* pdf, int N, uint32_t bin_cap, const uint32_t* bin,
                   const float* dir, uint32_t n, float* out, void* stream);

/* -------------------------------------------------------------------------
 * Learned proposal -- a project addition; the paper has no counterpart.
 * An MLP maps a bin origin's position and normal to a distribution over the
 * 32 x 32 cells of the same octahedral grid: features (78) = p^ = (p - lo) /
 * size, sin(2^k pi p^) and cos(2^k pi p^) for k = 0..11, and the normal;
 * layers 78 -> 64 -> 64 -> 64 -> 1024 with ReLU; softmax over the logits.
 * bfloat16 weights and activations, float32 accumulation on the tensor cores
 * (tcgen05), float32 master weights and Adam.  It is trained online on the
 * SVO-traced fields of guide_build_pdf with the loss KL(q || softmax(z)), q
 * the traced field normalised per bin; the traced PDF stays the fallback and
 * the reference the learned one is scored against.
 *
 * Parameters (WFPG_MLP_PARAMS float32, in this order): W1[64][80] (inputs
 * padded with two zero columns), b1[64], W2[64][64], b2[64], W3[64][64],
 * b3[64], W4[1024][64], b4[1024].
 */
#define WFPG_MLP_PARAMS 80064
typedef struct wfpg_mlp wfpg_mlp;

typedef struct wfpg_learned_params {
    float lo[3];   /* scene AABB lower corner (host) */
    float size;    /* scene AABB side */
    float eps;     /* floor added to every cell's probability before the CDF (keeps the PDF > 0) */
} wfpg_learned_params;

typedef struct wfpg_adam_params {
    float lr, beta1, beta2, eps;
    int update;    /* 0: compute the loss (and gradient) only, leave the weights */
} wfpg_adam_params;

/* mlp_create: device state for batches of up to max_batch samples; params is
 * a host array of WFPG_MLP_PARAMS floats (NULL: all zero).  Synchronises. */
WFPG_API int mlp_create(const float* params, uint32_t max_batch, void* stream, wfpg_mlp** out);
WFPG_API int mlp_destroy(wfpg_mlp* mlp);
/* copy the float32 master weights to a host array (synchronises) */
WFPG_API int mlp_get_params(const wfpg_mlp* mlp, float* params, void* stream);
/* status word (WFPG_STATUS_MMA_TIMEOUT), synchronises */
WFPG_API int mlp_status(wfpg_mlp* mlp, uint32_t* flags, int clear, void* stream);

/*
 * guide_learned_build_pdf -- the learned counterpart of guide_build_pdf (N =
 * 32): for each bin b < min(*n_bins_dev, bin_cap) (all bin_cap when NULL) the
 * MLP's distribution at the origin pos/nrm[origin_ray[b]] (row b when
 * origin_ray is NULL), plus eps per cell, becomes pdf / cdf_row / cdf_marg in
 * exactly the layout guide_sample and guide_eval_pdf read.  bin_cap <=
 * max_batch.
 */
WFPG_API int guide_learned_build_pdf(wfpg_mlp* mlp, const float* pos, const float* nrm,
                                     const uint32_t* origin_ray, const uint32_t* n_bins_dev,
                                     uint32_t bin_cap, const wfpg_learned_params* p, float* pdf,
                                     float* cdf_row, float* cdf_marg, void* stream);

/*
 * guide_learned_logits -- the network's logits for n samples (n <= max_batch):
 * logits[i][c] (device float [n][1024]) = the output layer's pre-softmax value
 * of cell c for the sample at pos/nrm[i], computed as guide_learned_build_pdf
 * computes it (bfloat16 operands, float32 accumulation).  For checking the
 * network against a reference and for callers that post-process the
 * distribution themselves.  Errors: null argument, n outside [1, max_batch]
 * (WFPG_ERR_CAPACITY), size <= 0.
 */
WFPG_API int guide_learned_logits(wfpg_mlp* mlp, const float* pos, const float* nrm, uint32_t n,
                                  const wfpg_learned_params* p, float* logits, void* stream);

/*
 * mlp_adam_step -- one Adam step (Kingma & Ba 2015) on the float32 master
 * weights with a caller-supplied gradient: grad is a device array of
 * WFPG_MLP_PARAMS floats in the parameter order above (e.g. the sum of several
 * guide_learned_train_step gradients).  Moments and step count are the
 * handle's, shared with guide_learned_train_step's own updates; the bfloat16
 * weight copies are refreshed.  opt->update is not read (the step is taken).
 * Errors: null argument; lr < 0, beta1 or beta2 outside [0, 1), eps < 0.
 */
WFPG_API int mlp_adam_step(wfpg_mlp* mlp, const float* grad, const wfpg_adam_params* opt, void* stream);

/*
 * guide_learned_train_step -- one step on n samples (n <= max_batch): pos/nrm
 * (xyz) of the sample points and target[n][1024], any non-negative field per
 * sample (normalised here; e.g. the pdf of guide_build_pdf at N = 32); target
 * must be 32-byte aligned (its rows are read with 32-byte loads).
 * Writes the mean KL to *loss_out and the gradient (WFPG_MLP_PARAMS floats)
 * to grad_out when they are not NULL (device pointers); with opt->update the
 * weights take one Adam step.
 * Errors: null argument or array, target not 32-byte aligned
 * (WFPG_ERR_INVALID_ARG); n = 0 or n > max_batch (WFPG_ERR_CAPACITY).
 */
WFPG_API int guide_learned_train_step(wfpg_mlp* mlp, const float* pos, const float* nrm, uint32_t n,
                                      const float* target, const wfpg_learned_params* p,
                                      const wfpg_adam_params* opt, float* loss_out, float* grad_out,
                                      void* stream);

/* -------------------------------------------------------------------------
 * Batched wavefront frame (a project addition; the paper launches every stage
 * of every depth from the host).  One frame is Alg. 1 for every pixel of a
 * pinhole camera, run entirely on the device:
 *   camera rays -> closest hits -> for each depth i = 1 .. max_depth:
 *     Partition-S (Alg. 2) of the live paths -> GuideRays (Alg. 3, fused:
 *     field + PDF/CDF in shared memory, then the bin's rays draw their next
 *     direction from alpha * guided + (1 - alpha) * cosine, exact density) ->
 *     Lambertian BSDF weight, closest hit, emission, Russian roulette from
 *     vertex rr_depth on (survival min(0.95, albedo)), order-preserving
 *     compaction of the survivors;
 *   then UpdateExitance: every vertex of every path gives one radiance
 *   record by Eq. 5 (zero when no emitter follows it), and svo_accumulate
 *   adds them and re-averages the tree.
 * Ray counts live in device memory between the stages, so the frame has no
 * host round trip and is replayed as one captured CUDA graph.  A frame index
 * in device memory advances after each frame and keys every random stream
 * (bins' origins, cell jitter, per-path uniforms: SplitMix64 counters).
 * The emitted radiance and albedo of a hit come from per-primitive device
 * arrays (quads first, then spheres, then triangles); a primitive with albedo
 * 0 ends a path.
 * Per-pixel sums of the path estimate and of its square accumulate over
 * frames (frame_image gives mean and variance of the mean).
 */
#define WFPG_FRAME_MAX_DEPTH 8

typedef struct wfpg_camera {
    float eye[3];
    float forward[3];   /* unit view direction */
    float up[3];        /* unit, orthogonal to forward */
    float vfov_deg;     /* vertical field of view */
    uint32_t width, height;
    /* Probe mode (radiance-field validation, Fig. 3): probe_pos != NULL replaces the pinhole.  It
       points to device float [height][3] probe points (copied at frame_create); pixel (x, y) is
       cell x of the side-probe_n concentric octahedral grid around point y (width must be
       probe_n^2) and its primary ray leaves point y in a uniformly random direction inside
       that cell, redrawn every frame.  The mean image is then the cell-averaged incident
       radiance at each probe (the cells have equal solid angle).  eye/forward/up/vfov unused. */
    const float* probe_pos;
    uint32_t probe_n;   /* 1 .. 1024 in probe mode */
} wfpg_camera;

typedef struct wfpg_frame_params {
    int max_depth;            /* guided bounces per path, 1 .. WFPG_FRAME_MAX_DEPTH */
    int rr_depth;             /* Russian roulette at vertices >= rr_depth (1 = first hit) */
    float alpha;              /* guided share of the one-sample mixture, [0, 1] */
    int l_min;                /* Partition-S */
    uint32_t c_ray;
    wfpg_guide_params guide;  /* N, eps, jitter, blur, t_skip, cos_weight, block, stage (seed/frame unused) */
    uint64_t seed;
    int update;               /* 1: UpdateExitance after each frame */
    int caster;               /* closest hits: 0 auto (SVO walk above 64 primitives), 1 every primitive, 2 SVO walk */
    int proposal;             /* guided part: 0 SVO-traced field (fused GuideRays), 1 learned MLP (N must be 32;
                                 frame_set_mlp first), 2 SVO-traced field times the BSDF (product guiding,
                                 Sec. 3.6; tables for up to 65,536 bins per depth, rays of further bins
                                 take the cosine branch) */
    int decay;                /* 1: the traced grid halves per depth (N, N/2, N/4, ..., at least 8), as the
                                 paper runs 128^2 .. 16^2 over four bounces */
    int combine;              /* image combination over frames (Eq. 7, weights h(i) of frame i = 1, 2, ...):
                                 0 constant, 1 linear (min(i, 5)), 2 quadratic (min(i, 5)^2), 3 one-two
                                 (1 then 2), 4 discard first (0 then 1), 5 PT first (frame 1 unguided,
                                 then constant) */
    int nee;                  /* 1: next-event estimation at every guided vertex (an emissive primitive by
                                 power, a uniform point on it, a shadow ray), combined with the mixture's
                                 samples by the power heuristic; Eq. 5 records include it, and a
                                 vertex's own record keeps its full emission while the vertices before
                                 it receive the MIS-weighted share */
} wfpg_frame_params;

typedef struct wfpg_frame wfpg_frame;

typedef struct wfpg_frame_stats {
    uint64_t frames;                                /* frames run since create / reset_image */
    uint32_t paths[WFPG_FRAME_MAX_DEPTH + 1];       /* live paths guided at depth i (last frame) */
    uint32_t bins[WFPG_FRAME_MAX_DEPTH + 1];        /* Partition-S bins at depth i (last frame) */
    uint32_t records;                               /* Eq. 5 records of the last frame */
    uint64_t guided_samples;                        /* sum of paths[] over all frames run */
    uint32_t status;                                /* the SVO's status bits */
    unsigned long long kernels_per_frame;           /* kernels in one captured frame */
} wfpg_frame_stats;

/* Creates a frame over an existing SVO (not owned; it must outlive the frame)
 * and scene (device pointers, not owned).  W x H x (WFPG_FRAME_MAX_DEPTH + 1)
 * must stay below 2^32 (32-bit record indices; about 477M pixels).  emission, albedo: device float
 * arrays, one per primitive.  Allocates the path state (about
 * 4 * W * H * (14 * (max_depth + 1) + 52) bytes, with the light-sample buffers) and builds the
 * light table from the scene (emissive primitives, chosen in proportion to emission x area).
 * Errors: invalid camera or parameters give WFPG_ERR_INVALID_ARG (probe mode: probe_n outside
 * 1 .. 1024 or width != probe_n^2); failed allocations WFPG_ERR_OOM.  Synchronises `stream`. */
WFPG_API int frame_create(wfpg_svo* svo, const wfpg_scene* scene, const float* emission, const float* albedo,
                          const wfpg_camera* cam, const wfpg_frame_params* p, wfpg_frame** out, void* stream);
WFPG_API int frame_destroy(wfpg_frame* f);
/* Runs n_frames frames on `stream` (asynchronous).  use_graph != 0 replays a
 * captured CUDA graph (captured on first use after create / set_params). */
WFPG_API int frame_run(wfpg_frame* f, uint32_t n_frames, int use_graph, void* stream);
/* Replaces the parameters (same max_depth or smaller; drops the graph). */
WFPG_API int frame_set_params(wfpg_frame* f, const wfpg_frame_params* p);
/* The MLP the learned proposal uses (not owned; NULL detaches).  Its bins per
 * depth are capped at min(its max_batch, the frame's bin capacity); rays of
 * bins past the cap take the cosine branch alone.  lp (copied): the scene box
 * and eps for guide_learned_build_pdf.  Drops the graph. */
WFPG_API int frame_set_mlp(wfpg_frame* f, wfpg_mlp* mlp, const wfpg_learned_params* lp);
WFPG_API int frame_get_params(const wfpg_frame* f, wfpg_frame_params* p);
/* Zeroes the per-pixel sums and the frame count. */
WFPG_API int frame_reset_image(wfpg_frame* f, void* stream);
/* mean[W*H] and var[W*H] (device, may be NULL): per-pixel combination of the
 * frames' path estimates, sum h(i) S_i / sum h(i) with the weights of
 * `combine`, and the (unweighted) variance of one frame's estimate (unbiased,
 * 0 when fewer than 2 frames). */
WFPG_API int frame_image(wfpg_frame* f, float* mean, float* var, void* stream);
/* Synchronises `stream` and reads the last frame's counts. */
WFPG_API int frame_stats(wfpg_frame* f, wfpg_frame_stats* out, void* stream);
/* Picks the grid side N among n_N candidates and the field kernel's tile
 * (block 64/128/256, staged or not): per N the fastest tile by frame time,
 * then the N with the least (mean per-pixel variance x frame time) over
 * `frames` frames.  The trial frames update the SVO as ordinary frames do.
 * Writes the choice into *chosen and applies it; resets the image. */
WFPG_API int frame_autotune(wfpg_frame* f, const int* N_candidates, int n_N, uint32_t frames,
                            wfpg_frame_params* chosen, float* ms_per_frame, void* stream);

/* Copies of internal buffers for inspection (tests): `what` selects one of
 * the WFPG_FRAME_BUF_* arrays; `bytes` must equal its size. */
enum {
    WFPG_FRAME_BUF_VT = 0,      /* float [max_depth+1][W*H]: throughput T(p_k) of vertex k */
    WFPG_FRAME_BUF_VLE = 1,     /* float [max_depth+1][W*H]: emitted radiance at vertex k */
    WFPG_FRAME_BUF_VPOS = 2,    /* float [max_depth+1][W*H][3] */
    WFPG_FRAME_BUF_VWO = 3,     /* float [max_depth+1][W*H][3]: unit direction toward the previous vertex */
    WFPG_FRAME_BUF_NV = 4,      /* u32 [W*H]: vertices of each path */
    WFPG_FRAME_BUF_REC_POS = 5, /* float [(max_depth+1)*W*H][3]; first `records` entries valid */
    WFPG_FRAME_BUF_REC_WOUT = 6,
    WFPG_FRAME_BUF_REC_L = 7,   /* float [(max_depth+1)*W*H] */
    WFPG_FRAME_BUF_REC_SRC = 8, /* u32 [(max_depth+1)*W*H]: k * W*H + path of each record */
    WFPG_FRAME_BUF_Q_POS = 9,   /* float [W*H][3]: positions of the last guided depth's queue */
    WFPG_FRAME_BUF_Q_NRM = 10,
    WFPG_FRAME_BUF_Q_U = 11,    /* float [W*H][3]: its uniforms */
    WFPG_FRAME_BUF_Q_DIR = 12,  /* float [W*H][3]: its sampled directions */
    WFPG_FRAME_BUF_Q_PDF = 13,  /* float [W*H]: their mixture densities */
    WFPG_FRAME_BUF_Q_PATH = 14, /* u32 [W*H]: path (pixel) of each queue slot */
    WFPG_FRAME_BUF_VNEE = 15,   /* float [max_depth+1][W*H]: MIS-weighted light sample per unit T(p_k) (nee) */
    WFPG_FRAME_BUF_NEE_DIR = 16, /* float [W*H][3]: last depth's light-sample direction per queue slot (nee) */
    WFPG_FRAME_BUF_NEE_PL = 17,  /* float [W*H]: its light-sampling density (solid angle; 0: none) */
    WFPG_FRAME_BUF_NEE_PM = 18,  /* float [W*H]: the mixture's density in that direction */
    WFPG_FRAME_BUF_NEE_L = 19,   /* float [W*H]: f cos Le / p_light of the sample (0: occluded) */
    WFPG_FRAME_BUF_VLW = 20,     /* float [max_depth+1][W*H]: emission as the previous vertex sees it (MIS-weighted) */
};
WFPG_API int frame_export(const wfpg_frame* f, int what, void* dst, size_t bytes, void* stream);

/* -------------------------------------------------------------------------
 * Measurement helper (renderer side; not part of the paper's method): the
 * closest hit of n rays (o + t d, t > tmin) against the scene's quads and
 * spheres.  t_out[i] = hit distance (-1 on a miss), prim_out[i] = primitive
 * (quads first, then spheres; 0xFFFFFFFF on a miss), nrm_out (xyz, may be
 * NULL) = geometric normal facing the ray.
 */
WFPG_API int wfpg_cast_rays(const wfpg_scene* scene, const float* o, const float* d, uint32_t n,
                            float tmin, float* t_out, uint32_t* prim_out, float* nrm_out, void* stream);
/* The same closest hit, with the scene's SVO (built from the same scene) as
 * the acceleration structure: the leaf-resolution walk of the cone march
 * visits the occupied leaves front to back and tests each leaf's fragment
 * list; empty blocks are skipped whole.  Hits agree with wfpg_cast_rays up
 * to a relative 1e-5 in t where two primitives are hit at nearly the same
 * distance. */
WFPG_API int wfpg_cast_rays_svo(const wfpg_svo* svo, const wfpg_scene* scene, const float* o, const float* d,
                                uint32_t n, float tmin, float* t_out, uint32_t* prim_out, float* nrm_out,
                                void* stream);

/* Measurement helper (not part of the paper's method): reads `bytes` of the
 * device buffer `buf` `reps` times through the L2 cache only (no L1
 * allocation), with `blocks` blocks of 512 threads; a buffer that fits in L2
 * gives the L2 read bandwidth the cone march is measured against.  *sink is
 * written only in a case the data makes unlikely (it keeps the loads).  buf
 * and bytes must be 16-byte aligned; reps, blocks >= 1. */
WFPG_API int wfpg_stream_read(const void* buf, size_t bytes, int reps, uint32_t* sink, int blocks, void* stream);

/* -------------------------------------------------------------------------
 * Inspection (used by tests; each synchronises `stream`).  Host buffers are
 * sized from svo_get_info: n_nodes entries (x2 for per-side arrays, x3 for
 * normals), n_frags fragment primitive ids, leaves + 1 fragment offsets.
 */
WFPG_API int svo_export(const wfpg_svo* svo, uint64_t* key, uint32_t* first_child, uint8_t* child_mask,
               uint32_t* parent, float* normal3, uint32_t* leaf_count, uint32_t* frag_off,
               uint32_t* frag_prim, void* stream);
WFPG_API int svo_export_exitance(const wfpg_svo* svo, uint64_t* acc_sum, uint32_t* acc_cnt,
                        uint64_t* tot_sum, uint32_t* tot_cnt, float* value, void* stream);

/* status word: host *flags receives the bits; clear != 0 zeroes it.
 * Synchronises `stream`. */
WFPG_API int wfpg_svo_status(wfpg_svo* svo, uint32_t* flags, int clear, void* stream);

WFPG_API const char* wfpg_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter, all threads and streams). */
WFPG_API unsigned long long wfpg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* WFPG_H */
