// Leaf-resolution walk helpers shared by the cone march (GuideRays) and the
// closest-hit caster: boundary times evaluated afresh from integer boundaries,
// and the cell a leaf-by-leaf DDA reaches on the other axes when the walk
// jumps over an empty block.
#pragma once
#include "common.cuh"

namespace wfpg {

// time of the crossing into cell j along one axis: boundary j when moving up,
// j + 1 when moving down; evaluated afresh from the integer boundary
__device__ __forceinline__ float cross_time(int j, bool up, float g, float inv) {
    return __fmul_rn(__fsub_rn((float)(up ? j : j + 1), g), inv);
}

// Index along one axis after every crossing strictly before time ts: the
// leaf-by-leaf walk's coordinate once it has passed all crossings < ts.
// May step one cell outside [0, res) (the ray left the grid before ts).
__device__ __forceinline__ int skip_before(int c, float g, float inv, float ts, int res) {
    if (inv == 0.0f) return c;
    const bool up = inv > 0.0f;
    for (int k = 0; k <= res; ++k) {
        const int nxt = up ? c + 1 : c - 1;
        if (!(cross_time(nxt, up, g, inv) < ts)) break;
        c = nxt;
        if (c < 0 || c >= res) break;
    }
    return c;
}

// Index along one axis that the leaf-by-leaf walk reaches at the crossing
// (tx, a): the last cell of the block [lo, lo + size) on this axis whose
// entry crossing comes before (tx, a) in (time, axis) order, starting from
// the current index c.  `before` says whether this axis precedes axis a.
__device__ __forceinline__ int advance_axis(int c, int lo, int size, float g, float inv, float ds, float tx,
                                            bool before) {
    if (inv == 0.0f || size == 1) return c;
    const int hi = lo + size - 1;
    const float p = g + tx * ds;
    const float fp = floorf(p);
    int j = (int)fp;
    // Fast path: the crossing tests below are monotone in the cell index and
    // agree with the real-number position up to relative roundings; their sum
    // stays under 1e-6 (|g| + |p| + 1) cells (four roundings of 2^-24 on the
    // crossing times, three on p).  When p lies at least that far inside a
    // cell, the tests would return floor(p) itself.
    const float m = 1e-6f * (fabsf(g) + fabsf(p) + 1.0f);
    const float f = p - fp;
    if (f >= m && f <= 1.0f - m && j >= lo && j <= hi && (inv > 0.0f ? j >= c : j <= c)) return j;
    j = max(lo, min(hi, j));  // otherwise the estimate is only a start; the checks decide
    if (inv > 0.0f) {
        j = max(j, c);
        while (j < hi) {
            const float tc = cross_time(j + 1, true, g, inv);
            if (tc < tx || (tc == tx && before)) ++j;
            else break;
        }
        while (j > c) {
            const float tc = cross_time(j, true, g, inv);
            if (tc < tx || (tc == tx && before)) break;
            --j;
        }
    } else {
        j = min(j, c);
        while (j > lo) {
            const float tc = cross_time(j - 1, false, g, inv);
            if (tc < tx || (tc == tx && before)) --j;
            else break;
        }
        while (j < c) {
            const float tc = cross_time(j, false, g, inv);
            if (tc < tx || (tc == tx && before)) break;
            ++j;
        }
    }
    return j;
}

}  // namespace wfpg
