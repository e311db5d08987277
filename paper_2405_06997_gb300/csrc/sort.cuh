// Device-wide scan and stable LSD radix sort used by the SVO builder and the
// binning step.  Scratch comes from a caller-provided workspace (Arena).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace wfpg {

// bump allocator over a caller-owned device buffer (256-byte aligned slices)
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    size_t used = 0;
    bool overflow = false;
    template <typename T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
        if (used + bytes > size) {
            overflow = true;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};
// byte count an Arena needs for `count` items of T
template <typename T>
inline size_t arena_bytes(size_t count) {
    return (count * sizeof(T) + 255) & ~(size_t)255;
}

constexpr int kScanBlock = 256, kScanItems = 8, kScanTile = kScanBlock * kScanItems;
constexpr int kSortBlock = 256, kSortItems = 16, kSortTile = kSortBlock * kSortItems;

size_t scan_workspace_bytes(uint32_t n);
// out[i] = sum of in[0..i) (out may alias in); *total_dev (if not null) = sum
void scan_exclusive(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* total_dev,
                    Arena& ws, cudaStream_t s);

size_t radix_sort_workspace_bytes(uint32_t n);
// Stable sort of keys (and values) by their low `bits` bits.  The sorted data
// ends in whichever buffer the returned pointers name.
void radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t n, int bits, Arena& ws,
                    cudaStream_t s, uint64_t** sorted);
// status (may be null): WFPG_STATUS_WAIT_TIMEOUT is or-ed into it when a wait of the one-sweep
// passes runs out (the result is then invalid)
void radix_sort_pairs_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                          uint32_t n, int bits, Arena& ws, cudaStream_t s, uint32_t** keys_out,
                          uint32_t** vals_out, uint32_t* status);

}  // namespace wfpg
