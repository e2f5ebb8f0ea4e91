// Bit-set helpers shared by the counting kernels: binary search among the
// candidates, the binary encoding of a root's induced sub-graph (Section 3.4)
// and the scan for the next member of a bit-set list.
#pragma once

#include <stdint.h>

namespace kc {

static constexpr uint32_t NONE = 0xFFFFFFFFu;

// First set bit of L at position >= from, scanning words up to hi (inclusive).
__device__ __forceinline__ uint32_t next_bit(const uint32_t* L, uint32_t from, uint32_t hi) {
    uint32_t w = from >> 5;
    if (w > hi) return NONE;
    uint32_t bits = L[w] & (0xFFFFFFFFu << (from & 31));
    while (bits == 0) {
        if (++w > hi) return NONE;
        bits = L[w];
    }
    return (w << 5) + (__ffs(bits) - 1);
}

// binary search of x in sorted s[lo, hi); returns index or NONE
__device__ __forceinline__ uint32_t find_sorted(const uint32_t* s, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint32_t y = s[mid];
        if (y == x) return mid;
        if (y < x) lo = mid + 1; else hi = mid;
    }
    return NONE;
}

// Rows of the induced sub-graph of cand[0, d): bit j of row i iff cand[j] in
// N+(cand[i]).  One warp per row; lanes take 32 consecutive entries of
// N+(cand[i]) at a time and binary-search them among cand[i+1 .. d).
template <int NT>
__device__ void build_bitmap(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ col, const uint32_t* cand,
                             uint32_t d, uint32_t W, uint32_t* bm) {
    for (uint32_t x = threadIdx.x; x < d * W; x += NT) bm[x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t last = cand[d - 1];
    for (uint32_t i = warp; i < d; i += NT / 32) {
        const uint32_t x = cand[i];
        const uint32_t b = rp[x], e = rp[x + 1];
        uint32_t* row = bm + (size_t)i * W;
        for (uint32_t j0 = b; j0 < e; j0 += 32) {
            uint32_t j = j0 + lane;
            uint32_t y = j < e ? col[j] : NONE;
            if (y != NONE && y <= last) {
                uint32_t pos = find_sorted(cand, i + 1, d, y);
                if (pos != NONE) atomicOr(&row[pos >> 5], 1u << (pos & 31));
            }
            if (__shfl_sync(0xffffffffu, y, 31) >= last) break;  // the rest of the row lies beyond cand
        }
    }
    __syncthreads();
}

}  // namespace kc
