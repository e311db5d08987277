// CPU ORACLE -- TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
//
// Positional binning (Sec. 3.4, Alg. 2 "Partition-S") and the choice of each
// bin's field origin (Sec. 3 "Implementation": a randomly chosen hit point of
// the bin, drawn anew every iteration).
#include <algorithm>
#include <numeric>

#include "oracle_internal.h"

namespace orc {

// Partition-S.  Levels are numbered from the root = 0 (the paper counts the
// root as level 1).
//  1. every ray descends to the deepest existing node holding its position
//     and increments that node's ray counter (DescendLeaf + AtomicAdd);
//  2. for the levels D down to l_min, a node's total T is its own counter plus
//     its children's totals; it is marked when T >= c_ray or l == l_min;
//  3. every ray ascends from its node to the first marked node, itself
//     included (AscendAndFindMarked); a ray whose node lies above l_min keeps
//     its own node;
//  4. bins are numbered by ascending global node id; rays are stably
//     partitioned by bin (Partition).
// Returns the number of bins.
uint32_t partition_s(const Svo& s, const float* pos, size_t n, int l_min, uint32_t c_ray,
                     uint32_t* bin_of_ray, uint32_t* ray_order, std::vector<uint32_t>& bin_offset) {
    const int D = s.D;
    if (l_min < 0) l_min = 0;
    if (l_min > D) l_min = D;
    const uint32_t N = s.num_nodes();
    std::vector<uint32_t> node_of(n), count(N, 0), total(N, 0);
    std::vector<uint8_t> mark(N, 0);
    for (size_t i = 0; i < n; ++i) {
        node_of[i] = s.deepest(pos + 3 * i);
        count[node_of[i]] += 1;
    }
    for (int l = D; l >= l_min; --l) {
        for (uint32_t node = s.level_off[l]; node < s.level_off[l + 1]; ++node) {
            uint32_t T = count[node];
            if (l < D) {
                int m = __builtin_popcount(s.child_mask[node]);
                for (int c = 0; c < m; ++c) T += total[s.first_child[node] + c];
            }
            total[node] = T;
            mark[node] = (T >= c_ray || l == l_min) ? 1 : 0;
        }
    }
    std::vector<uint32_t> bin_node(n);
    std::vector<uint8_t> used(N, 0);
    for (size_t i = 0; i < n; ++i) {
        uint32_t node = node_of[i];
        if (s.level_of(node) >= l_min) {
            while (!mark[node]) node = s.parent[node];
        }
        bin_node[i] = node;
        used[node] = 1;
    }
    std::vector<uint32_t> rank(N, NONE);
    uint32_t nb = 0;
    for (uint32_t node = 0; node < N; ++node)
        if (used[node]) rank[node] = nb++;
    for (size_t i = 0; i < n; ++i) bin_of_ray[i] = rank[bin_node[i]];
    std::vector<uint32_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](uint32_t a, uint32_t b) { return bin_of_ray[a] < bin_of_ray[b]; });
    std::copy(idx.begin(), idx.end(), ray_order);
    bin_offset.assign(nb + 1, 0);
    for (size_t i = 0; i < n; ++i) bin_offset[bin_of_ray[i] + 1] += 1;
    for (uint32_t b = 0; b < nb; ++b) bin_offset[b + 1] += bin_offset[b];
    return nb;
}

// Stand-in binning for frame-scale workloads whose bins follow a given length
// mix: rays are keyed by their leaf cell at level min(6, D) (Morton order)
// and the octant of their normal, stably sorted by that key, and the sorted
// sequence is cut into runs of the given sizes; run j is bin j.
// Returns the number of bins, or 0 if the sizes do not add up to n or one is 0.
uint32_t partition_runs(const Svo& s, const float* pos, const float* nrm, size_t n,
                        const uint32_t* sizes, uint32_t nb, uint32_t* bin_of_ray,
                        uint32_t* ray_order, std::vector<uint32_t>& bin_offset) {
    uint64_t total = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        if (sizes[b] == 0) return 0;
        total += sizes[b];
    }
    if (total != n) return 0;
    const int D = s.D;
    const int q = D < 6 ? D : 6;
    std::vector<uint64_t> key(n);
    for (size_t i = 0; i < n; ++i) {
        uint32_t c[3];
        for (int a = 0; a < 3; ++a)
            c[a] = (uint32_t)grid_index(pos[3 * i + a], s.lo[a], s.scale, D) >> (D - q);
        const float* N = nrm + 3 * i;
        uint32_t oct = (N[0] < 0.0f ? 1u : 0u) | (N[1] < 0.0f ? 2u : 0u) | (N[2] < 0.0f ? 4u : 0u);
        key[i] = (morton(c[0], c[1], c[2]) << 3) | oct;
    }
    std::vector<uint32_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return key[a] < key[b]; });
    bin_offset.assign(nb + 1, 0);
    for (uint32_t b = 0; b < nb; ++b) bin_offset[b + 1] = bin_offset[b] + sizes[b];
    for (uint32_t b = 0; b < nb; ++b)
        for (uint32_t k = bin_offset[b]; k < bin_offset[b + 1]; ++k) bin_of_ray[idx[k]] = b;
    std::copy(idx.begin(), idx.end(), ray_order);
    return nb;
}

// SelectOrigin: bin b takes the ray at position floor(u * n_b) of its run,
// u the 24-bit uniform of (seed, frame, b); computed exactly as
// (u24 * n_b) >> 24.
void select_origins(const uint32_t* ray_order, const std::vector<uint32_t>& bin_offset,
                    uint32_t nb, uint64_t seed, uint32_t frame, uint32_t* origin_ray) {
    for (uint32_t b = 0; b < nb; ++b) {
        uint64_t cnt = bin_offset[b + 1] - bin_offset[b];
        uint64_t u = rng_u24(purpose_seed(seed, PURPOSE_ORIGIN), bin_stream(frame, b), 0);
        uint64_t k = (u * cnt) >> 24;
        origin_ray[b] = ray_order[bin_offset[b] + k];
    }
}

}  // namespace orc
