// CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, step-by-step CPU restatement of the wavefront path-guiding
// hot path (Yalciner & Akyuz, "Path Guiding for Wavefront Path Tracing").
// Only the tests, the smoke check and the benchmark's CPU-baseline leg may
// load it.  It shares no code with the CUDA library: it is written from the
// paper's description, in the paper's order, with no blocking or fusion.
//
// Floating point: every step whose result decides an integer (voxel
// occupancy, the traversed leaf, the cone level, the side, the sampled cell)
// is computed in IEEE binary32 with one rounding per written operation
// (built with -ffp-contract=off), because that is the precision the kernels
// take those decisions in; the paper does not fix a precision.  Sphere
// occupancy is decided in binary64.
#pragma once
#include <cstdint>
#include <cstddef>
#include <vector>

namespace orc {

// ---------------------------------------------------------------------------
// Counter-based random numbers: the SplitMix64 output function of Steele, Lea
// and Flood (OOPSLA 2014) applied to a (seed, stream, counter) triple.
//   key   = mix64(seed XOR stream * GAMMA)
//   value = mix64(key + (counter + 1) * GAMMA)
// The 24 high bits give a uniform on the 2^-24 lattice of [0, 1).
inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}
constexpr uint64_t GAMMA = 0x9e3779b97f4a7c15ULL;
inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t counter) {
    uint64_t key = mix64(seed ^ (stream * GAMMA));
    return mix64(key + (counter + 1) * GAMMA);
}
inline uint32_t rng_u24(uint64_t seed, uint64_t stream, uint64_t counter) {
    return (uint32_t)(rng_u64(seed, stream, counter) >> 40);
}
inline float rng_unit(uint64_t seed, uint64_t stream, uint64_t counter) {
    return (float)rng_u24(seed, stream, counter) * 0x1p-24f;
}
// purposes folded into the seed so that streams never collide
constexpr uint64_t PURPOSE_ORIGIN = 0;
constexpr uint64_t PURPOSE_JITTER = 1;
inline uint64_t purpose_seed(uint64_t seed, uint64_t purpose) { return seed * 4 + purpose; }
inline uint64_t bin_stream(uint32_t frame, uint32_t bin) {
    return ((uint64_t)frame << 32) | (uint64_t)bin;
}

// ---------------------------------------------------------------------------
// Morton key of leaf coordinates: bit i of x goes to bit 3i, of y to 3i+1, of
// z to 3i+2 (x least significant), the Z-order used for sorting voxels before
// building the hierarchy (Sec. 3.2).
inline uint64_t morton(uint32_t x, uint32_t y, uint32_t z) {
    uint64_t k = 0;
    for (int i = 0; i < 21; ++i) {
        k |= (uint64_t)((x >> i) & 1u) << (3 * i);
        k |= (uint64_t)((y >> i) & 1u) << (3 * i + 1);
        k |= (uint64_t)((z >> i) & 1u) << (3 * i + 2);
    }
    return k;
}
inline void morton_decode(uint64_t k, uint32_t* x, uint32_t* y, uint32_t* z) {
    *x = *y = *z = 0;
    for (int i = 0; i < 21; ++i) {
        *x |= (uint32_t)((k >> (3 * i)) & 1u) << i;
        *y |= (uint32_t)((k >> (3 * i + 1)) & 1u) << i;
        *z |= (uint32_t)((k >> (3 * i + 2)) & 1u) << i;
    }
}

// world coordinate -> leaf index on one axis: floor((x - lo) * scale) clamped
// to [0, 2^D - 1] (NaN -> 0)
inline int32_t grid_index(float x, float lo, float scale, int D) {
    float g = (x - lo) * scale;
    if (!(g >= 0.0f)) return 0;
    int32_t res = 1 << D;
    if (g >= (float)res) return res - 1;
    return (int32_t)g;
}

constexpr uint32_t NONE = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// The sparse voxel octree, level-major: level l (root = 0, leaves = D) holds
// the sorted unique Morton prefixes of the occupied leaves; the global node id
// is level_off[l] + index in level.
struct Svo {
    int D = 0;
    float lo[3] = {0, 0, 0};
    float S = 1;
    float scale = 1;                                 // 2^D / S
    std::vector<std::vector<uint64_t>> keys;         // keys[l]
    std::vector<uint32_t> level_off;                 // D + 2 entries
    std::vector<uint32_t> first_child, parent;       // global ids
    std::vector<uint8_t> child_mask;
    std::vector<uint32_t> leaf_count;
    std::vector<float> normal;                       // 3 per node
    std::vector<uint32_t> frag_off;                  // leaves + 1 (fragments per leaf)
    std::vector<uint32_t> frag_prim;
    // radiant exitance, 2 sides per node
    std::vector<uint64_t> acc_sum, tot_sum;
    std::vector<uint32_t> acc_cnt, tot_cnt;
    std::vector<float> value;

    uint32_t num_nodes() const { return level_off.empty() ? 0 : level_off[D + 1]; }
    int level_of(uint32_t node) const {
        for (int l = 0; l <= D; ++l)
            if (node < level_off[l + 1]) return l;
        return -1;
    }
    // global id of the node with this prefix at level l, or NONE
    uint32_t find(int l, uint64_t prefix) const;
    // deepest existing node whose cube contains the point p (Alg. 2 DescendLeaf)
    uint32_t deepest(const float p[3]) const;
};

Svo* build_svo(const float* quads, int nq, const float* spheres, int ns, const float* tris, int nt,
               const float lo[3], float S, int D);

// k-means with k = 2 over weighted unit vectors (Sec. 3.2, Fig. 2)
void kmeans2(const float* n, const float* w, int m, float out[3]);

// directional helpers (Clarberg 2008 concentric octahedral map, own trig)
float poly_sin(float x);
float poly_cos(float x);
float poly_atan01(float q);
void octa_decode(float u, float v, float out[3]);
void octa_encode(const float d[3], float* u, float* v);

struct TraceResult {
    int hit;
    uint64_t leaf_key;
    float t_entry;
    int level;
    uint32_t node;
    int side;
    float value;
    uint32_t steps;   // leaf cells the DDA entered
    uint32_t blocks;  // maximal empty blocks and leaves passed (when counted)
};
TraceResult trace_cell(const Svo& s, const float o[3], const float d[3], float t_skip,
                       float omega, int cos_weight, bool count_blocks = false);

}  // namespace orc
