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

// position of the m-th (0-based) bit of L strictly above a (one thread)
__device__ __forceinline__ uint32_t select_above(const uint32_t* L, uint32_t a, uint32_t m, uint32_t W) {
    uint32_t lo = a + 1;
    for (uint32_t w = lo >> 5; w < W; ++w) {
        uint32_t x = L[w];
        if (w == (lo >> 5)) x &= 0xFFFFFFFFu << (lo & 31);
        const uint32_t c = __popc(x);
        if (m < c) return (w << 5) + __fns(x, 0, m + 1);
        m -= c;
    }
    return NONE;
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

// The entries y <= last of the sorted DAG row col[b, e), handed to f(y) by
// the 32 lanes of a warp.  Each lane loads two 16-byte quads per round (a
// warp covers 256 entries per round with all loads in flight), and the scan
// stops after the round whose final entry exceeds last.  The row array must
// be 16-byte aligned and readable up to the quad holding entry e - 1.
template <class F>
__device__ __forceinline__ void scan_row(const uint32_t* __restrict__ col, uint32_t b, uint32_t e, uint32_t last,
                                         int lane, F&& f) {
    const uint4* col4 = reinterpret_cast<const uint4*>(col);
    const uint32_t qend = (e + 3) >> 2;
    for (uint32_t q0 = b >> 2; q0 < qend; q0 += 64) {
        const uint32_t qa = q0 + lane, qb = qa + 32;
        uint4 va = make_uint4(NONE, NONE, NONE, NONE), vb = va;
        if (qa < qend) va = __ldg(col4 + qa);
        if (qb < qend) vb = __ldg(col4 + qb);
        const uint32_t ja = qa << 2, jb = qb << 2;
        const uint32_t ya[4] = {va.x, va.y, va.z, va.w};
        const uint32_t yb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (ja + c >= b && ja + c < e && ya[c] <= last) f(ya[c]);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (jb + c >= b && jb + c < e && yb[c] <= last) f(yb[c]);
        const uint32_t tail = (jb + 3 < e) ? vb.w : NONE;
        if (__shfl_sync(0xffffffffu, tail, 31) >= last) break;  // the rest of the row lies beyond last
    }
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
        uint32_t* row = bm + (size_t)i * W;
        scan_row(col, __ldg(rp + x), __ldg(rp + x + 1), last, lane, [&](uint32_t y) {
            const uint32_t pos = find_sorted(cand, i + 1, d, y);
            if (pos != NONE) atomicOr(&row[pos >> 5], 1u << (pos & 31));
        });
    }
    __syncthreads();
}

// Open-addressing table of the candidates' positions, for the membership
// test of the bitmap build: 2^tbits 16-bit slots holding position + 1
// (0 = empty), linear probing from a multiplicative hash of the vertex id.
// Most tested ids are not candidates, and at a load of at most 1/4 most of
// those misses end at the first, empty, slot.
__host__ __device__ __forceinline__ uint32_t hash_slot(uint32_t y, uint32_t tbits) {
    return (y * 0x9E3779B1u) >> (32 - tbits);
}

__host__ __device__ __forceinline__ uint32_t hash_bits_for(uint32_t d) {
    uint32_t b = 6;
    while ((1u << b) < 4 * d) ++b;
    return b;
}

// Candidate filter beside the table: one bit per slot of a larger hash
// range, set for every candidate (bit hash_slot(y, fbits)).  A clear bit
// proves that y is not a candidate; a set bit (a candidate, or a false
// positive at a rate of at most 1/32) sends y to the table.  At least 32
// slots per candidate, at least 1,024.
__host__ __device__ __forceinline__ uint32_t filter_bits_for(uint32_t d) {
    uint32_t b = 10;
    while ((1u << b) < 32 * d) ++b;
    return b;
}

__host__ __device__ __forceinline__ uint32_t filter_words(uint32_t d) { return (1u << filter_bits_for(d)) >> 5; }

// 32-bit words of the table and its filter for candidate sets up to d
// (both grow with d, so a smaller set fits the space of a larger one)
__host__ __device__ __forceinline__ uint32_t hash_table_words(uint32_t d) {
    return (1u << hash_bits_for(d)) / 2 + filter_words(d);
}

// The entries y of the sorted DAG row col[b, e) whose filter bit is set
// (bit hash_slot(y, fbits) of filt), handed to f(y) by the 32 lanes of a
// warp.  Each lane loads two 16-byte quads per round (256 entries per warp
// round, all loads in flight) and tests its 8 entries without branching;
// only the entries that pass are handed to f, one after another.  Filtering
// first keeps the lanes of a warp together: the data-dependent work (the
// exact lookup of about one entry in eight) runs as one loop per round
// instead of once per entry.  The scan stops after the round whose final
// entry exceeds last.  The row array must be 16-byte aligned and readable up
// to the quad holding entry e - 1; filt is read at words below 2^fbits / 32.
template <class F>
__device__ __forceinline__ void scan_row_filtered(const uint32_t* __restrict__ col, uint32_t b, uint32_t e,
                                                  uint32_t last, int lane, const uint32_t* filt, uint32_t fbits,
                                                  F&& f) {
    const uint4* col4 = reinterpret_cast<const uint4*>(col);
    const uint32_t qend = (e + 3) >> 2;
    const uint32_t len = e - b;
    for (uint32_t q0 = b >> 2; q0 < qend; q0 += 64) {
        const uint32_t qa = q0 + lane, qb = qa + 32;
        uint4 va = make_uint4(NONE, NONE, NONE, NONE), vb = va;
        if (qa < qend) va = __ldg(col4 + qa);
        if (qb < qend) vb = __ldg(col4 + qb);
        const uint32_t y[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
        // offsets of the quads' first entries within the row; entries before
        // b wrap to large values, so one unsigned compare keeps [b, e)
        const uint32_t ta = (qa << 2) - b, tb = (qb << 2) - b;
        uint32_t pend = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t t = (c < 4 ? ta : tb) + (uint32_t)(c & 3);
            const uint32_t hf = hash_slot(y[c], fbits);
            const uint32_t bit = (filt[hf >> 5] >> (hf & 31)) & 1u;
            pend |= (t < len ? bit : 0u) << c;
        }
        while (pend) {
            const int c = __ffs(pend) - 1;
            pend &= pend - 1;
            uint32_t yc = y[0];
#pragma unroll
            for (int x = 1; x < 8; ++x) yc = (c == x) ? y[x] : yc;
            f(yc);
        }
        const uint32_t tail = ((qb << 2) + 3 < e) ? vb.w : NONE;
        if (__shfl_sync(0xffffffffu, tail, 31) >= last) break;  // the rest of the row lies beyond last
    }
}

// Same rows as build_bitmap, with the table and filter above instead of
// binary search.  tab: hash_table_words(d) words: 2^tbits 16-bit slots
// (tbits from hash_bits_for(d)), then the filter (filter_bits_for(d) bits);
// d < 65535.
template <int NT>
__device__ void build_bitmap_hashed(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                    const uint32_t* cand, uint32_t d, uint32_t W, uint32_t* bm, uint32_t* tabw,
                                    uint32_t tbits) {
    const uint32_t T = 1u << tbits, mask = T - 1;
    const uint32_t fbits = filter_bits_for(d);
    uint16_t* tab = reinterpret_cast<uint16_t*>(tabw);
    uint32_t* filt = tabw + T / 2;
    for (uint32_t x = threadIdx.x; x < d * W; x += NT) bm[x] = 0;
    for (uint32_t x = threadIdx.x; x < T / 2 + filter_words(d); x += NT) tabw[x] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < d; i += NT) {
        const uint32_t y = cand[i];
        uint32_t h = hash_slot(y, tbits);
        while (atomicCAS(&tab[h], (unsigned short)0, (unsigned short)(i + 1)) != 0) h = (h + 1) & mask;
        const uint32_t hf = hash_slot(y, fbits);
        atomicOr(&filt[hf >> 5], 1u << (hf & 31));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t last = cand[d - 1];
    // row bounds of the warp's next row are loaded while it scans this one
    uint32_t nb = 0, ne = 0;
    if (warp < d) {
        nb = __ldg(rp + cand[warp]);
        ne = __ldg(rp + cand[warp] + 1);
    }
    for (uint32_t i = warp; i < d; i += NT / 32) {
        const uint32_t b = nb, e = ne;
        if (i + NT / 32 < d) {
            const uint32_t x2 = cand[i + NT / 32];
            nb = __ldg(rp + x2);
            ne = __ldg(rp + x2 + 1);
        }
        uint32_t* row = bm + (size_t)i * W;
        scan_row_filtered(col, b, e, last, lane, filt, fbits, [&](uint32_t y) {
            uint32_t h = hash_slot(y, tbits);
            for (;;) {
                const uint32_t p = tab[h];
                if (p == 0) break;
                if (cand[p - 1] == y) {
                    atomicOr(&row[(p - 1) >> 5], 1u << ((p - 1) & 31));
                    break;
                }
                h = (h + 1) & mask;
            }
        });
    }
    __syncthreads();
}

}  // namespace kc
