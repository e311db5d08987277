// Library-side state of one sparse voxel octree (the wfpg_svo handle).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

struct wfpg_svo {
    int device = 0;
    int D = 0;
    float lo[3] = {0, 0, 0};
    float S = 1.0f;
    float scale = 1.0f;                       // 2^D / S in binary32
    uint32_t n_nodes = 0;
    uint32_t n_frags = 0;
    uint32_t level_off[WFPG_MAX_DEPTH + 2] = {0};
    // topology (level-major, global ids)
    wfpg::Node* node = nullptr;               // first child + child mask
    uint32_t* parent = nullptr;
    uint64_t* key = nullptr;                  // Morton prefix of each node at its level
    uint32_t* leaf_count = nullptr;
    float4* normal = nullptr;                 // (nx, ny, nz, 0)
    uint8_t* route = nullptr;                 // bit0/bit1: parent side taking this node's side 0/1
    // top index: for each level l <= top_levels - 1, a dense grid over that level's cells
    // (x fastest) holding (L << 28) | node, node = the deepest existing node at a level
    // L <= l containing the cell (empty when top_levels == 0)
    uint32_t* top = nullptr;
    int top_levels = 0;
    uint32_t top_off[8] = {0};
    // occupancy bitmaps of the levels top_levels .. D (only when D <= kOccMaxDepth): level
    // l's bit k is set iff the node of Morton key k exists at level l; words of level l
    // start at occ_off[l]
    uint32_t* occ = nullptr;
    uint64_t occ_off[WFPG_MAX_DEPTH + 2] = {0};
    uint32_t* frag_off = nullptr;             // leaves + 1
    uint32_t* frag_prim = nullptr;            // n_frags
    // radiant exitance, two sides per node
    unsigned long long* acc_sum = nullptr;    // records added at this node
    uint32_t* acc_cnt = nullptr;
    unsigned long long* tot_sum = nullptr;    // own + children (inner nodes)
    uint32_t* tot_cnt = nullptr;
    float2* value = nullptr;
    uint32_t* status = nullptr;               // WFPG_STATUS_* bits (word 0); word 1: bin_next
    uint32_t* bin_next = nullptr;             // next bin for the field kernel's CTAs (reset per launch)
};

namespace wfpg {
void svo_free_arrays(wfpg_svo* s);
}
