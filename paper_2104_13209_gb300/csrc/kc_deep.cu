// Graph-orientation counting (Fig. 2) for larger k: the search tree below a
// root is deep, and almost all of its nodes sit at the last levels, where
// the candidate lists are short (on R-MAT scale 20 at k = 6, 98 % of the
// size-5 nodes have at most 128 candidates, while the root bitmaps are up to
// 20 words wide).
//
// A root r with more than 32 candidates is taken by a block, which builds
// the binary encoding of its induced sub-graph (Section 3.4) as in the
// k <= 4 kernel.  The block's warps claim tasks of the root:
//   vertex-centric (VC): root edges r -> C[t]; the node below is row t;
//   edge-centric (EC):   root triangles (r, C[t], C[u]) with u in row t; the
//                        node below is row t & row u.
// A node is a candidate list L (a bitmap over the root's candidates) and the
// number of vertices still to choose, rem:
//   rem == 1:   count += |L|
//   rem == 2:   count += the edges of the sub-graph induced by L
//               (lanes take members j of L, each sums popc(L & row_j))
//   |L| <= 128: the sub-graph induced by L is re-encoded (Section 2.4 allows
//               extraction at any level) as |L| rows of 1, 2 or 4 words: row a
//               of the new encoding has bit b iff member b is an
//               out-neighbour of member a, gathered 32 bits at a time with a
//               warp ballot.  The lanes then split its edges (a, b) as tasks
//               and each walks the rest of the subtree alone on 1-4 word
//               lists, with an explicit per-lane stack.
//   otherwise:  the warp steps through the members v of L (ascending, while
//               enough remain) and descends into L & row_v; the lists of the
//               wide levels are kept in a per-warp stack.
// Roots with at most 32 candidates run in warp mode (kc_dfs.cuh).  Counts are
// exact 128-bit sums, reduced as in the k <= 4 kernel.
#include <algorithm>

#include "kc_dfs.cuh"

namespace kc {

static constexpr int DW = 8;                 // warps per block
static constexpr int DBLOCK = DW * 32;
static constexpr uint32_t CMAX = 128;        // members of a re-encoded node
static constexpr int LANE_DEPTH = 32;        // per-lane stack levels (k <= 36)
static constexpr uint32_t DEEP_MAX_K = 36;

// Per-warp shared memory.
struct DeepWarp {
    uint32_t T[CMAX * 4];      // re-encoded rows, nw words each
    uint32_t pre[CMAX + 4];    // exclusive prefix of the rows' popcounts (task numbering)
    uint16_t pos[CMAX];        // members' positions among the root's candidates
    uint32_t next;             // next unclaimed lane task
    uint32_t pad[3];
};
static_assert(sizeof(DeepWarp) % 16 == 0, "per-warp areas keep 16-byte alignment");

struct DeepParams {
    CountParams base;
    int ec;
    uint32_t wp;                 // words per bitmap row (a multiple of 4)
    uint32_t wide_levels;        // wide stack levels per warp
    uint32_t* task_total;        // per big root: its number of tasks (EC: edges of its sub-graph), 0 = unknown
    unsigned long long* pv;      // per-vertex counts, library numbering (per-vertex variant)
    uint32_t n;                  // vertices
};

// Per-vertex counts (PV).  A vertex gains, for every counted clique that
// holds it, one: the root gains its tree's count, a vertex on the path to a
// node gains the count of the node's subtree, and below a node whose last
// two vertices are chosen together (the edges of the sub-graph induced by
// L) a member j of L gains its degree in that sub-graph, popc(L & row_j) +
// popc(L & column_j), read from the encoding and its transpose.
struct PvCtx {
    unsigned long long* pvc;  // block: per root candidate position, [d] = the root
    const uint32_t* bmT;      // transposed root bitmap (row j = the candidates with j in their row)
    uint32_t* TT;             // warp: transposed re-encoded rows
    unsigned long long* pvm;  // warp: gains of the re-encoded members
    uint32_t* scand;          // warp: a small root's candidates
    uint32_t ncand;           // the current root's candidates (pvc has ncand + 1 entries)
};

// Per-warp shared memory of the per-vertex variant (after the wide stacks).
struct DeepWarpPv {
    uint32_t TT[CMAX * 4];
    unsigned long long pvm[CMAX];
    uint32_t scand[32];
};
static_assert(sizeof(DeepWarpPv) % 16 == 0, "per-warp areas keep 16-byte alignment");

__device__ __forceinline__ void pv_add(unsigned long long* p, unsigned long long x, const Ctl* ctl) {
    if (x == 0) return;
    const unsigned long long old = atomicAdd(p, x);
    if (old + x < old) atomicOr((unsigned*)&ctl->flags, (unsigned)KC_FLAG_VERTEX_OVERFLOW);
}

// pv_add to entry idx of an array of `bound` entries (bounds-checked)
__device__ __forceinline__ void pv_add_at(unsigned long long* base, uint32_t idx, uint32_t bound, unsigned long long x,
                                          const Ctl* ctl, unsigned code) {
    if (x == 0) return;
    if (!in_bounds(const_cast<Ctl*>(ctl), idx, bound, code)) return;
    pv_add(base + idx, x, ctl);
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// Lane-level walk over a re-encoded node of nw words per row (nw = 1, 2, 4)
// ---------------------------------------------------------------------------
template <int NW>
struct Mask {
    uint32_t w[NW];
};

template <int NW>
__device__ __forceinline__ Mask<NW> mask_and(const Mask<NW>& a, const uint32_t* row) {
    Mask<NW> r;
    if (NW == 4) {
        const uint4 x = *reinterpret_cast<const uint4*>(row);
        r.w[0] = a.w[0] & x.x;
        r.w[1 % NW] = a.w[1 % NW] & x.y;
        r.w[2 % NW] = a.w[2 % NW] & x.z;
        r.w[3 % NW] = a.w[3 % NW] & x.w;
    } else if (NW == 2) {
        const uint2 x = *reinterpret_cast<const uint2*>(row);
        r.w[0] = a.w[0] & x.x;
        r.w[1 % NW] = a.w[1 % NW] & x.y;
    } else {
        r.w[0] = a.w[0] & row[0];
    }
    return r;
}

template <int NW>
__device__ __forceinline__ uint32_t mask_popc(const Mask<NW>& a) {
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) c += __popc(a.w[i]);
    return c;
}

// Lowest member of a (NONE if empty), removed from a.
template <int NW>
__device__ __forceinline__ uint32_t mask_pop(Mask<NW>& a) {
#pragma unroll
    for (int i = 0; i < NW; ++i)
        if (a.w[i]) {
            const uint32_t b = __ffs(a.w[i]) - 1;
            a.w[i] &= a.w[i] - 1;
            return (uint32_t)i * 32 + b;
        }
    return NONE;
}

// popc(J & row) over words i..NW-1 (row: a re-encoded row whose member
// lies in word i, so its words below i are zero)
template <int NW, int I>
__device__ __forceinline__ uint32_t popc_from(const Mask<NW>& J, const uint32_t* row) {
    uint32_t c = 0;
    if (NW == 4 && I <= 1) {
        const uint4 x = *reinterpret_cast<const uint4*>(row);
        if (I == 0) c += __popc(J.w[0] & x.x);
        c += __popc(J.w[1 % NW] & x.y) + __popc(J.w[2 % NW] & x.z) + __popc(J.w[3 % NW] & x.w);
    } else if (NW == 4 && I == 2) {
        const uint2 x = *reinterpret_cast<const uint2*>(row + 2);
        c += __popc(J.w[2 % NW] & x.x) + __popc(J.w[3 % NW] & x.y);
    } else if (NW == 2 && I == 0) {
        const uint2 x = *reinterpret_cast<const uint2*>(row);
        c += __popc(J.w[0] & x.x) + __popc(J.w[1 % NW] & x.y);
    } else {
        c += __popc(J.w[I % NW] & row[I % NW]);  // the last word
    }
    return c;
}

// sum over the members v of J in word I of popc(J & T[v]) (one lane)
template <int NW, int I>
__device__ __forceinline__ uint32_t edges_in_word(const Mask<NW>& J, const uint32_t* T) {
    uint32_t s = 0, bits = J.w[I % NW];
    while (bits) {
        const uint32_t v = I * 32 + (__ffs(bits) - 1);
        bits &= bits - 1;
        s += popc_from<NW, I>(J, T + (size_t)v * NW);
    }
    return s;
}

// Edges of the sub-graph induced by J (rows T, nw words each): members in
// word i only need the row words from i on (rows are upper triangular).
// PV: each member gains its degree in that sub-graph (out-neighbours from
// T, in-neighbours from the transpose TT).
template <int NW, bool PV>
__device__ __forceinline__ unsigned long long lane_edges(Mask<NW> J, const uint32_t* T, const PvCtx& X, const Ctl* ctl,
                                                         unsigned long long& words) {
    if (PV) {
        const Mask<NW> J0 = J;
        unsigned long long s = 0;
        for (;;) {
            const uint32_t v = mask_pop<NW>(J);
            if (v == NONE) break;
            const uint32_t out = mask_popc<NW>(mask_and<NW>(J, T + (size_t)v * NW));
            s += out;
            const uint32_t in = mask_popc<NW>(mask_and<NW>(J0, X.TT + (size_t)v * NW));
            pv_add_at(X.pvm, v, CMAX, out + in, ctl, 201u);
            words += 2 * NW;
        }
        return s;
    }
    uint32_t s = edges_in_word<NW, 0>(J, T);
    if (NW > 1) s += edges_in_word<NW, 1>(J, T);
    if (NW > 2) {
        s += edges_in_word<NW, 2>(J, T);
        s += edges_in_word<NW, 3>(J, T);
    }
    words += (unsigned long long)mask_popc<NW>(J) * NW;
    return s;
}

// rem-cliques of the sub-graph induced by J0 (rem >= 3), one lane alone.
// PV: the vertex chosen at each level gains the count of its subtree
// (pending sums flushed when the level moves on).
template <int NW, bool PV>
__device__ unsigned long long lane_walk_nw(const Ctl* ctl, Mask<NW> J0, uint32_t rem0, const uint32_t* T,
                                           const PvCtx& X, unsigned long long& words) {
    Mask<NW> stk[LANE_DEPTH];
    uint32_t cv[PV ? LANE_DEPTH : 1];
    unsigned long long pend[PV ? LANE_DEPTH : 1];
    unsigned long long acc = 0, tot = 0;
    int l = 0;
    stk[0] = J0;
    if (PV) pend[0] = 0;
    uint32_t steps = 0;
    auto flush = [&](int lv) {
        if (PV && pend[lv]) {
            pv_add_at(X.pvm, cv[lv], CMAX, pend[lv], ctl, 202u);
            if (lv > 0) pend[lv - 1] += pend[lv];
            else tot += pend[lv];
            pend[lv] = 0;
        }
    };
    for (;;) {
        Mask<NW>& J = stk[l];
        const uint32_t rem = rem0 - l;
        if (mask_popc<NW>(J) < rem) {
            if (PV) flush(l);
            if (l == 0) break;
            --l;
            continue;
        }
        if ((++steps & 1023u) == 0 && timed_out(ctl)) break;
        const uint32_t v = mask_pop<NW>(J);
        if (PV) {
            flush(l);
            cv[l] = v;
        }
        const Mask<NW> C = mask_and<NW>(J, T + (size_t)v * NW);
        words += NW;
        const uint32_t c = mask_popc<NW>(C);
        const uint32_t need = rem - 1;
        if (c < need) continue;
        if (need == 2) {
            const unsigned long long e = lane_edges<NW, PV>(C, T, X, ctl, words);
            acc += e;
            if (PV) pend[l] += e;
        } else {
            stk[++l] = C;
            if (PV) pend[l] = 0;
        }
    }
    (void)tot;
    return acc;
}

// The transpose of the re-encoded rows (X.TT: row b = the members a < b with
// b in row a) and cleared member gains, for the per-vertex variant.
template <int NW>
__device__ __forceinline__ void transpose_small(const DeepWarp& dw, const PvCtx& X, uint32_t m) {
    const int lane = threadIdx.x & 31;
    for (uint32_t b = 0; b < m; ++b) {
#pragma unroll
        for (int c = 0; c < NW; ++c) {
            const uint32_t a = (uint32_t)c * 32 + lane;
            const bool bit = a < m && a < b && ((dw.T[a * NW + (b >> 5)] >> (b & 31)) & 1u);
            const uint32_t w = __ballot_sync(0xffffffffu, bit);
            if (lane == c) X.TT[b * NW + c] = w;
        }
    }
    for (uint32_t a = lane; a < m; a += 32) X.pvm[a] = 0;
    __syncwarp();
}

// rem-cliques (rem >= 2) of the re-encoded sub-graph on m vertices held in
// dw.T, by the 32 lanes of the warp; returns this lane's share of the count
// (also added to acc).  rem == 2: lanes take rows; rem == 3: lanes take rows
// and count each row's edges; rem == 4: lanes claim rows and count the edges
// below each of their edges; rem >= 5: lanes claim the edges (a, b) of the
// sub-graph one at a time and walk below a & b.
// PV: X.pvm[a] receives the number of counted cliques holding member a.
template <int NW, bool PV>
__device__ unsigned long long warp_small(const Ctl* ctl, DeepWarp& dw, const PvCtx& X, uint32_t m, uint32_t rem,
                                         Acc& acc) {
    const int lane = threadIdx.x & 31;
    const uint32_t* T = dw.T;
    if (PV) transpose_small<NW>(dw, X, m);
    unsigned long long s = 0;
    if (rem == 3 && !PV) {
        // lanes claim rows, the heavy first ones first (rows are upper
        // triangular); a row's triangles with it as the smallest member
        if (lane == 0) dw.next = 0;
        __syncwarp();
        for (;;) {
            const uint32_t a = atomicAdd(&dw.next, 1u);
            if (a >= m || timed_out(ctl)) break;
            Mask<NW> R;
#pragma unroll
            for (int i = 0; i < NW; ++i) R.w[i] = T[a * NW + i];
            s += lane_edges<NW, false>(R, T, X, ctl, acc.words);
        }
        acc.add(s);
        __syncwarp();
        return s;
    }
    if (rem <= 3) {
        for (uint32_t a = lane; a < m; a += 32) {
            Mask<NW> R;
#pragma unroll
            for (int i = 0; i < NW; ++i) R.w[i] = T[a * NW + i];
            if (rem == 2) {
                const uint32_t out = mask_popc<NW>(R);
                s += out;
                acc.words += NW;
                if (PV) {
                    Mask<NW> C;
#pragma unroll
                    for (int i = 0; i < NW; ++i) C.w[i] = X.TT[a * NW + i];
                    pv_add_at(X.pvm, a, CMAX, out + mask_popc<NW>(C), ctl, 203u);
                }
            } else {
                // triangles with a as the smallest member
                Mask<NW> B = R;
                unsigned long long t = 0;
                for (;;) {
                    const uint32_t b = mask_pop<NW>(B);
                    if (b == NONE) break;
                    t += mask_popc<NW>(mask_and<NW>(R, T + (size_t)b * NW));
                    acc.words += NW;
                }
                s += t;
                if (PV) {
                    // ... plus those with a as the middle or the largest member
                    Mask<NW> C;
#pragma unroll
                    for (int i = 0; i < NW; ++i) C.w[i] = X.TT[a * NW + i];
                    Mask<NW> A = C;
                    for (;;) {
                        const uint32_t x = mask_pop<NW>(A);
                        if (x == NONE) break;
                        t += mask_popc<NW>(mask_and<NW>(R, T + (size_t)x * NW));
                        t += mask_popc<NW>(mask_and<NW>(C, T + (size_t)x * NW));
                        acc.words += 2 * NW;
                    }
                    pv_add_at(X.pvm, a, CMAX, t, ctl, 204u);
                }
            }
        }
        acc.add(s);
        __syncwarp();
        return s;
    }
    if (rem == 4) {
        // lanes claim rows; below each edge (a, b) of a row, count the edges of a & b
        if (lane == 0) dw.next = 0;
        __syncwarp();
        for (;;) {
            const uint32_t a = atomicAdd(&dw.next, 1u);
            if (a >= m || timed_out(ctl)) break;
            Mask<NW> R;
#pragma unroll
            for (int i = 0; i < NW; ++i) R.w[i] = T[a * NW + i];
            Mask<NW> B = R;
            unsigned long long sa = 0;
            for (;;) {
                const uint32_t b = mask_pop<NW>(B);
                if (b == NONE) break;
                const Mask<NW> J = mask_and<NW>(R, T + (size_t)b * NW);
                acc.words += NW;
                if (mask_popc<NW>(J) >= 2) {
                    const unsigned long long e = lane_edges<NW, PV>(J, T, X, ctl, acc.words);
                    sa += e;
                    if (PV) pv_add_at(X.pvm, b, CMAX, e, ctl, 205u);
                }
            }
            s += sa;
            if (PV) pv_add_at(X.pvm, a, CMAX, sa, ctl, 206u);
        }
        acc.add(s);
        __syncwarp();
        return s;
    }
    // rem >= 5: edge tasks, numbered row by row
    uint32_t carry = 0;
    for (uint32_t a0 = 0; a0 < m; a0 += 32) {
        const uint32_t a = a0 + lane;
        uint32_t c = 0;
        if (a < m) {
#pragma unroll
            for (int i = 0; i < NW; ++i) c += __popc(T[a * NW + i]);
        }
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (a < m) dw.pre[a] = carry + incl - c;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        dw.pre[m] = carry;
        dw.next = 0;
    }
    __syncwarp();
    const uint32_t total = carry;
    const uint32_t rem2 = rem - 2;  // vertices still to choose below an edge task
    for (;;) {
        const uint32_t t = atomicAdd(&dw.next, 1u);
        if (t >= total || timed_out(ctl)) break;
        uint32_t lo = 0, hi = m;  // the row a with pre[a] <= t < pre[a + 1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (dw.pre[mid] <= t) lo = mid; else hi = mid;
        }
        uint32_t r = t - dw.pre[lo];  // the r-th member of row lo
        const uint32_t* Ra = T + (size_t)lo * NW;
        uint32_t b = NONE;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const uint32_t x = Ra[i], c = __popc(x);
            if (b == NONE) {
                if (r < c) b = (uint32_t)i * 32 + __fns(x, 0, (int)r + 1);
                else r -= c;
            }
        }
        Mask<NW> A;
#pragma unroll
        for (int i = 0; i < NW; ++i) A.w[i] = Ra[i];
        const Mask<NW> J = mask_and<NW>(A, T + (size_t)b * NW);
        acc.words += NW;
        const uint32_t c = mask_popc<NW>(J);
        if (c < rem2) continue;
        unsigned long long e;
        if (rem2 == 1) e = c;
        else if (rem2 == 2) e = lane_edges<NW, PV>(J, T, X, ctl, acc.words);
        else e = lane_walk_nw<NW, PV>(ctl, J, rem2, T, X, acc.words);
        s += e;
        if (PV) {
            pv_add_at(X.pvm, lo, CMAX, e, ctl, 207u);
            pv_add_at(X.pvm, b, CMAX, e, ctl, 208u);
        }
    }
    acc.add(s);
    __syncwarp();
    return s;
}

// ---------------------------------------------------------------------------
// Warp-level steps on a list L over the root's candidates (rows of wp words)
// ---------------------------------------------------------------------------

// members of L (m <= CMAX) into dw.pos, in ascending order
__device__ __forceinline__ void list_members(const uint32_t* L, uint32_t wp, DeepWarp& dw) {
    const int lane = threadIdx.x & 31;
    uint32_t carry = 0;
    for (uint32_t x0 = 0; x0 < wp; x0 += 32) {
        const uint32_t x = x0 + lane;
        const uint32_t bits0 = x < wp ? L[x] : 0u;
        const uint32_t c = __popc(bits0);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t o = carry + incl - c;
        if (x < wp && wp <= CMAX + 4) dw.pre[x] = o;  // word prefix, for reencode_rows
        uint32_t bits = bits0;
        while (bits) {
            if (o < CMAX) dw.pos[o] = (uint16_t)((x << 5) + (__ffs(bits) - 1));
            ++o;
            bits &= bits - 1;
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
}

// Re-encode the sub-graph induced by L (m <= CMAX members, word prefixes of L
// in dw.pre, wp <= CMAX + 4) into dw.T with NW words per row, one lane per
// row: each member of row pos[a] & L at word x and bit i becomes bit
// pre[x] + popc(L[x] below i) of row a.  The work follows the sub-graph's
// edges, not m^2.
template <int NW>
__device__ __forceinline__ void reencode_rows(const uint32_t* bm, const uint32_t* L, uint32_t wp, uint32_t m,
                                              DeepWarp& dw) {
    const int lane = threadIdx.x & 31;
    for (uint32_t a = lane; a < m; a += 32) {
        const uint32_t pa = dw.pos[a];
        const uint32_t* row = bm + (size_t)pa * wp;
        uint32_t o0 = 0, o1 = 0, o2 = 0, o3 = 0;
        for (uint32_t x = pa >> 5; x < wp; ++x) {
            const uint32_t lx = L[x];
            uint32_t v = row[x] & lx;
            if (!v) continue;
            const uint32_t base = dw.pre[x];
            while (v) {
                const uint32_t i = __ffs(v) - 1;
                v &= v - 1;
                const uint32_t idx = base + __popc(lx & ((1u << i) - 1u));
                const uint32_t bit = 1u << (idx & 31);
                if (idx < 32) o0 |= bit;
                else if (idx < 64) o1 |= bit;
                else if (idx < 96) o2 |= bit;
                else o3 |= bit;
            }
        }
        dw.T[a * NW] = o0;
        if (NW > 1) dw.T[a * NW + 1 % NW] = o1;
        if (NW > 2) {
            dw.T[a * NW + 2 % NW] = o2;
            dw.T[a * NW + 3 % NW] = o3;
        }
    }
    __syncwarp();
}

// Re-encode the sub-graph induced by L (m <= CMAX members) into dw.T with NW
// words per row: bit b of row a iff pos[b] is in row pos[a] of bm (32 bits
// at a time by warp ballots; for rows too wide for reencode_rows).
template <int NW>
__device__ __forceinline__ void reencode(const uint32_t* bm, uint32_t wp, uint32_t m, DeepWarp& dw) {
    const int lane = threadIdx.x & 31;
    uint32_t pb[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        const uint32_t b = (uint32_t)c * 32 + lane;
        pb[c] = b < m ? (uint32_t)dw.pos[b] : 0u;
    }
    for (uint32_t a = 0; a < m; ++a) {
        const uint32_t* row = bm + (size_t)dw.pos[a] * wp;
#pragma unroll
        for (int c = 0; c < NW; ++c) {
            const uint32_t b = (uint32_t)c * 32 + lane;
            const bool bit = b < m && b > a && ((row[pb[c] >> 5] >> (pb[c] & 31)) & 1u);
            const uint32_t w = __ballot_sync(0xffffffffu, bit);
            if (lane == c) dw.T[a * NW + c] = w;
        }
    }
    __syncwarp();
}

// Edges of the sub-graph induced by L (rows of bm, wp words each): lanes take
// the words of L round-robin, and for each member j in them sum
// popc(L & row_j) from j's word on.  PV: j gains its degree in the sub-graph,
// the in-neighbours read from the transposed bitmap (row j of bmT, words up
// to j's).
template <bool PV>
__device__ __forceinline__ unsigned long long wide_edges(const uint32_t* L, const uint32_t* bm, uint32_t wp,
                                                         uint32_t lo, const PvCtx& X, const Ctl* ctl,
                                                         unsigned long long& words) {
    const int lane = threadIdx.x & 31;
    unsigned long long s = 0;
    for (uint32_t w = lo + lane; w < wp; w += 32) {
        uint32_t bits = L[w];
        while (bits) {
            const uint32_t j = (w << 5) + (__ffs(bits) - 1);
            bits &= bits - 1;
            const uint32_t* rj = bm + (size_t)j * wp;
            uint32_t c = 0;
            uint32_t x = w;
            for (; x < wp && (x & 3u) != 0; ++x) c += __popc(L[x] & rj[x]);
            for (; x + 4 <= wp; x += 4) {
                const uint4 a = *reinterpret_cast<const uint4*>(L + x);
                const uint4 r = *reinterpret_cast<const uint4*>(rj + x);
                c += __popc(a.x & r.x) + __popc(a.y & r.y) + __popc(a.z & r.z) + __popc(a.w & r.w);
            }
            for (; x < wp; ++x) c += __popc(L[x] & rj[x]);
            s += c;
            words += wp - w;
            if (PV) {
                const uint32_t* tj = X.bmT + (size_t)j * wp;
                uint32_t in = 0;
                for (uint32_t y = lo; y <= w; ++y) in += __popc(L[y] & tj[y]);
                words += w - lo + 1;
                pv_add_at(X.pvc, j, X.ncand + 1, (unsigned long long)c + in, ctl, 209u);
            }
        }
    }
    return s;
}

// wide_edges for m <= CMAX members listed in dw.pos: the lanes take the
// members, first and last alternately (row lengths fall with the position),
// so every lane scans about the same number of words.
template <bool PV>
__device__ __forceinline__ unsigned long long wide_edges_listed(const uint32_t* L, const uint32_t* bm, uint32_t wp,
                                                                uint32_t lo, uint32_t m, const DeepWarp& dw,
                                                                const PvCtx& X, const Ctl* ctl,
                                                                unsigned long long& words) {
    const int lane = threadIdx.x & 31;
    unsigned long long s = 0;
    for (uint32_t i = lane; i < m; i += 32) {
        const uint32_t jj = (i & 1u) ? m - 1 - (i >> 1) : (i >> 1);
        const uint32_t j = dw.pos[jj];
        const uint32_t w = j >> 5;
        const uint32_t* rj = bm + (size_t)j * wp;
        uint32_t c = 0;
        uint32_t x = w;
        for (; x < wp && (x & 3u) != 0; ++x) c += __popc(L[x] & rj[x]);
        for (; x + 4 <= wp; x += 4) {
            const uint4 a = *reinterpret_cast<const uint4*>(L + x);
            const uint4 r = *reinterpret_cast<const uint4*>(rj + x);
            c += __popc(a.x & r.x) + __popc(a.y & r.y) + __popc(a.z & r.z) + __popc(a.w & r.w);
        }
        for (; x < wp; ++x) c += __popc(L[x] & rj[x]);
        s += c;
        words += wp - w;
        if (PV) {
            const uint32_t* tj = X.bmT + (size_t)j * wp;
            uint32_t in = 0;
            for (uint32_t y = lo; y <= w; ++y) in += __popc(L[y] & tj[y]);
            words += w - lo + 1;
            pv_add_at(X.pvc, j, X.ncand + 1, (unsigned long long)c + in, ctl, 209u);
        }
    }
    return s;
}

// popc of L over the warp
__device__ __forceinline__ uint32_t warp_popc(const uint32_t* L, uint32_t lo, uint32_t wp) {
    const int lane = threadIdx.x & 31;
    uint32_t c = 0;
    for (uint32_t w = lo + lane; w < wp; w += 32) c += __popc(L[w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

// ---------------------------------------------------------------------------
// Sharing the wide levels between the warps of a block.  A root's giant
// subtrees (hubs of a dense core) would otherwise run on one warp while the
// block's other warps wait.  A warp walking a wide level donates the upper
// half of the remaining children of its shallowest splittable level when
// warps are idle: the frame holds a copy of the level's list, the cursor
// and end of the donated range, the members from the cursor on (for the size
// bound), the number of vertices still to choose, and (per-vertex counts)
// the path positions whose gains include the frame's count.
// ---------------------------------------------------------------------------
static constexpr int DQCAP = 8;
static constexpr int DPATH = LANE_DEPTH + 4;
// A warp waiting for a frame gives up after this long (the donors finish
// their own work, so leaving is always safe).
static constexpr unsigned long long DEEP_IDLE_NS = 2000000000ull;

struct DeepSteal {
    unsigned idle;     // warps waiting for a frame (or trying to take one)
    unsigned active;   // warps still in the session
    unsigned queued;   // frames ready
    unsigned left_pool;  // warps that stopped waiting after DEEP_IDLE_NS
    unsigned state[DQCAP];  // 0 empty, 1 being written, 2 ready, 3 being read
    unsigned meta[DQCAP][4];  // cursor, end, rem, members after the cursor
    unsigned npath[DQCAP];
    unsigned path[DQCAP][DPATH];
};

// Lane-indexed warp-uniform array: lane i holds entry i.
__device__ __forceinline__ uint32_t lget(uint32_t reg, int i) { return __shfl_sync(0xffffffffu, reg, i); }
__device__ __forceinline__ unsigned long long lget64(unsigned long long reg, int i) {
    return __shfl_sync(0xffffffffu, reg, i);
}

// members of L in (a, b) (positions), over the warp
__device__ __forceinline__ uint32_t warp_range_popc(const uint32_t* L, uint32_t a, uint32_t b, uint32_t wp) {
    const int lane = threadIdx.x & 31;
    uint32_t c = 0;
    const uint32_t lo = a + 1;  // a = NONE wraps to 0
    if (lo < b) {
        const uint32_t w0 = lo >> 5, w1 = min((b - 1) >> 5, wp - 1);
        for (uint32_t w = w0 + lane; w <= w1; w += 32) {
            uint32_t x = L[w];
            if (w == w0) x &= 0xFFFFFFFFu << (lo & 31);
            if (w == ((b - 1) >> 5)) x &= 0xFFFFFFFFu >> (31 - ((b - 1) & 31));
            c += __popc(x);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

// Where a walk starts: either a node (L, lo, m, rem) to analyse, or a donated
// frame (a level with list L whose children after `cursor` and before `end`
// remain; `cnt` members after the cursor; rem for the level's node).
struct WalkStart {
    const uint32_t* L;
    uint32_t lo, m, rem;
    bool frame;
    uint32_t cursor, end, cnt;
};

// The walk of the root's tree from s.  stk: the warp's wide stack (levels x
// wp words).  path / npath: positions (among the root's candidates) on the
// path above s, warp-uniform (lane i holds entry i); with PV every count
// below s is also their gain (the root's gain is added by the caller).
// PV: returns the count below s (the same on every lane); the members of the
// nodes below and the vertices chosen at the wide levels gain theirs.
template <bool PV>
__device__ unsigned long long deep_walk(const DeepParams& D, const uint32_t* bm, const WalkStart& s0, uint32_t* stk,
                                        DeepWarp& dw, const PvCtx& X, Acc& acc, DeepSteal* ss, uint32_t* qwords,
                                        uint32_t path_reg, uint32_t npath) {
    const int lane = threadIdx.x & 31;
    const uint32_t wp = D.wp;
    const Ctl* ctl = D.base.ctl;
    // wide levels, lane-indexed: cursor, end of the range, members after the
    // cursor, pending count (PV); level l's list is Ls0 (l = 0) or stk + (l - 1) wp
    uint32_t cur_r = 0, end_r = 0, left_r = 0;
    unsigned long long pend_r = 0;
    const uint32_t* Ls0 = s0.L;
    unsigned long long tot = 0;
    int l = -1;
    const uint32_t rem0 = s0.rem;
    const uint32_t* L = s0.L;
    uint32_t lo = s0.lo, m = s0.m, rem = s0.rem;
    uint32_t steps = 0;
    bool analyse = !s0.frame;
    if (s0.frame) {
        l = 0;
        if (lane == 0) {
            cur_r = s0.cursor;
            end_r = s0.end;
            left_r = s0.cnt;
            pend_r = 0;
        }
    }
    auto lst = [&](int lv) -> const uint32_t* { return lv == 0 ? Ls0 : stk + (size_t)(lv - 1) * wp; };
    // PV: the vertex chosen at level lv gains its subtree; so do the levels above
    auto flush = [&](int lv) {
        if (!PV) return;
        const unsigned long long p = lget64(pend_r, lv);
        if (p == 0) return;
        const uint32_t cv = lget(cur_r, lv);  // every lane takes part in the shuffle
        if (lane == 0) pv_add_at(X.pvc, cv, X.ncand + 1, p, ctl, 212u);
        if (lv > 0) {
            if (lane == lv - 1) pend_r += p;
        } else {
            tot += p;
        }
        if (lane == lv) pend_r = 0;
    };
    for (;;) {
        if (analyse) {
            bool descend = false;
            unsigned long long c_node = 0;  // PV: the node's count when it is finished here
            if (rem == 1) {
                if (lane == 0) acc.add(m);
                c_node = m;
                if (PV) {
                    for (uint32_t w = lo + lane; w < wp; w += 32) {
                        uint32_t bits = L[w];
                        while (bits) {
                            pv_add_at(X.pvc, (w << 5) + (__ffs(bits) - 1), X.ncand + 1, 1ull, ctl, 210u);
                            bits &= bits - 1;
                        }
                    }
                }
            } else if (rem == 2) {
                unsigned long long e;
                if (m <= CMAX) {
                    list_members(L, wp, dw);
                    e = wide_edges_listed<PV>(L, bm, wp, lo, m, dw, X, ctl, acc.words);
                    __syncwarp();
                } else {
                    e = wide_edges<PV>(L, bm, wp, lo, X, ctl, acc.words);
                }
                acc.add(e);
                if (PV) c_node = warp_sum64(e);
            } else if (m <= CMAX) {
                list_members(L, wp, dw);
                unsigned long long e;
                const bool rows = wp <= CMAX + 4;
                if (m <= 32) {
                    if (rows) reencode_rows<1>(bm, L, wp, m, dw); else reencode<1>(bm, wp, m, dw);
                    e = warp_small<1, PV>(ctl, dw, X, m, rem, acc);
                } else if (m <= 64) {
                    if (rows) reencode_rows<2>(bm, L, wp, m, dw); else reencode<2>(bm, wp, m, dw);
                    e = warp_small<2, PV>(ctl, dw, X, m, rem, acc);
                } else {
                    if (rows) reencode_rows<4>(bm, L, wp, m, dw); else reencode<4>(bm, wp, m, dw);
                    e = warp_small<4, PV>(ctl, dw, X, m, rem, acc);
                }
                if (PV) {
                    c_node = warp_sum64(e);
                    for (uint32_t a = lane; a < m; a += 32) pv_add_at(X.pvc, dw.pos[a], X.ncand + 1, X.pvm[a], ctl, 211u);
                    __syncwarp();
                }
            } else if (l + 1 < (int)D.wide_levels && l + 1 < LANE_DEPTH) {
                descend = true;
            } else if (lane == 0) {
                atomicOr((unsigned*)&ctl->flags, (unsigned)KC_FLAG_INTERNAL);  // cannot happen: depth < k
            }
            if (PV && !descend) {
                if (l >= 0) {
                    if (lane == l) pend_r += c_node;
                } else {
                    tot += c_node;
                }
            }
            if (descend) {
                ++l;
                if (l == 0) Ls0 = L;
                if (lane == l) {
                    cur_r = lo * 32 - 1;  // before the first member (NONE when lo == 0)
                    end_r = NONE;
                    left_r = m;
                    pend_r = 0;
                }
            }
        }
        analyse = true;
        // next child of the deepest wide level that still has one
        for (;;) {
            if (l < 0) return tot;
            const uint32_t r = rem0 - (uint32_t)l;  // rem of level l's node
            if (lget(left_r, l) < r) {
                flush(l);
                --l;
                continue;
            }
            if ((++steps & 63u) == 0) {
                {
                    int to = lane == 0 ? (int)timed_out(ctl) : 0;
                    if (__shfl_sync(0xffffffffu, to, 0)) return tot;
                }
                // donate the upper half of the shallowest level with two or more children left
                int want = 0;
                if (lane == 0) want = *(volatile unsigned*)&ss->idle > 0 && *(volatile unsigned*)&ss->queued < DQCAP;
                if (__shfl_sync(0xffffffffu, want, 0)) {
                    for (int lv = 0; lv <= l; ++lv) {
                        const uint32_t* Lv = lst(lv);
                        const uint32_t cv = lget(cur_r, lv), ev = lget(end_r, lv);
                        const uint32_t nr = warp_range_popc(Lv, cv, ev, wp);
                        if (nr < 2 || lget(left_r, lv) < rem0 - (uint32_t)lv) continue;
                        uint32_t q = NONE, split = NONE;
                        if (lane == 0) {
                            split = select_above(Lv, cv, nr / 2, wp);
                            for (uint32_t x = 0; x < DQCAP; ++x)
                                if (*(volatile unsigned*)&ss->state[x] == 0 && atomicCAS(&ss->state[x], 0u, 1u) == 0u) {
                                    q = x;
                                    break;
                                }
                        }
                        q = __shfl_sync(0xffffffffu, q, 0);
                        split = __shfl_sync(0xffffffffu, split, 0);
                        if (q == NONE || split == NONE) break;
                        uint32_t* dst = qwords + (size_t)q * wp;
                        for (uint32_t w = lane; w < wp; w += 32) dst[w] = Lv[w];
                        const uint32_t tc = warp_range_popc(Lv, split - 1, NONE, wp);
                        // path of the donated children: the path above this walk, then the
                        // vertices chosen at levels 0 .. lv - 1
                        const uint32_t np = npath + (uint32_t)lv;
                        if (PV) {
                            if (lane < (int)npath) ss->path[q][lane] = path_reg;
                            const uint32_t cr = cur_r;  // lane i: level i's vertex
                            if (lane < lv) ss->path[q][npath + lane] = cr;
                        }
                        if (lane == 0) {
                            ss->meta[q][0] = split - 1;
                            ss->meta[q][1] = ev;
                            ss->meta[q][2] = rem0 - (uint32_t)lv;
                            ss->meta[q][3] = tc;
                            ss->npath[q] = np;
                        }
                        __syncwarp();
                        if (lane == 0) {
                            __threadfence_block();
                            atomicExch(&ss->state[q], 2u);
                            atomicAdd(&ss->queued, 1u);
                        }
                        if (lane == lv) end_r = split;
                        break;
                    }
                }
            }
            const uint32_t* Ll = lst(l);
            uint32_t v = next_bit(Ll, lget(cur_r, l) + 1, wp - 1);  // cur = NONE wraps to 0
            if (v != NONE && v >= lget(end_r, l)) v = NONE;
            flush(l);
            if (v == NONE) {
                --l;
                continue;
            }
            if (lane == l) {
                cur_r = v;
                --left_r;
            }
            uint32_t* C = stk + (size_t)l * wp;
            const uint32_t clo = (v + 1) >> 5;
            const uint32_t* rv = bm + (size_t)v * wp;
            __syncwarp();
            uint32_t c = 0;
            for (uint32_t w = lane; w < wp; w += 32) {
                const uint32_t x = w >= clo ? (Ll[w] & rv[w]) : 0u;
                C[w] = x;
                c += __popc(x);
            }
            acc.words += (lane == 0) ? (wp - clo) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            __syncwarp();
            if (c < r - 1) continue;
            L = C;
            lo = clo;
            m = c;
            rem = r - 1;
            break;
        }
    }
}

// A warp out of tasks: take a donated frame (copied to own, wp words; meta
// and path to *f), or wait until one appears or every warp of the block is
// idle.  Returns false when the session is over for this warp.
__device__ bool deep_steal(const Ctl* ctl, DeepSteal* ss, const uint32_t* qwords, uint32_t wp, uint32_t* own,
                           WalkStart* f, uint32_t* path_reg, uint32_t* npath) {
    const int lane = threadIdx.x & 31;
    uint32_t q = NONE;
    if (lane == 0) {
        atomicAdd(&ss->idle, 1u);
        const unsigned long long t0 = globaltimer_ns();
        bool done = false;
        for (uint32_t it = 0;; ++it) {
            if (*(volatile unsigned*)&ss->queued > 0) {
                atomicSub(&ss->idle, 1u);  // trying to take work: no longer idle
                for (uint32_t x = 0; x < DQCAP; ++x)
                    if (*(volatile unsigned*)&ss->state[x] == 2u && atomicCAS(&ss->state[x], 2u, 3u) == 2u) {
                        q = x;
                        break;
                    }
                if (q != NONE) {
                    atomicSub(&ss->queued, 1u);
                    break;
                }
                atomicAdd(&ss->idle, 1u);
            }
            if (*(volatile unsigned*)&ss->idle == *(volatile unsigned*)&ss->active &&
                *(volatile unsigned*)&ss->queued == 0) {
                done = true;
                break;
            }
            if ((it & 255u) == 255u) {
                if (timed_out(ctl) || globaltimer_ns() - t0 > DEEP_IDLE_NS) {
                    // leave the pool: the warps still walking finish their own frames
                    atomicSub(&ss->idle, 1u);
                    atomicSub(&ss->active, 1u);
                    atomicAdd(&ss->left_pool, 1u);
                    done = true;
                    break;
                }
            }
            __nanosleep(128);
        }
        (void)done;
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q == NONE) return false;
    __threadfence_block();
    const uint32_t* src = qwords + (size_t)q * wp;
    for (uint32_t w = lane; w < wp; w += 32) own[w] = src[w];
    f->L = own;
    f->frame = true;
    f->cursor = ss->meta[q][0];
    f->end = ss->meta[q][1];
    f->rem = ss->meta[q][2];
    f->cnt = ss->meta[q][3];
    f->lo = 0;
    f->m = 0;
    *npath = ss->npath[q];
    *path_reg = lane < (int)*npath ? ss->path[q][lane] : 0u;
    __syncwarp();
    if (lane == 0) atomicExch(&ss->state[q], 0u);
    return true;
}

// ---------------------------------------------------------------------------

struct DeepShared {
    uint32_t slot;
    uint32_t task;      // next unclaimed task of a root no other block joins
    uint32_t total;     // the root's number of tasks
};

// Pick the next big root: own a new one while any is left, then join roots
// whose published task count shows enough unclaimed tasks.
__device__ uint32_t deep_next_slot(const DeepParams& D, WorkCtl* wc, int& phase) {
    const CountParams& P = D.base;
    if (timed_out(P.ctl)) return NONE;
    if (phase == 0) {
        const uint32_t s = atomicAdd(&wc->root_cursor, 1u);
        if (s < P.n_big) return s;
        phase = 1;
    }
    if (P.help_min == 0) return NONE;
    uint32_t lo = atomicAdd(&wc->help_lo, 0u);
    for (uint32_t probes = 0; lo < P.n_big && probes < 4096; ++lo, ++probes) {
        const uint32_t total = atomicAdd(&D.task_total[lo], 0u);
        if (total == 0) continue;  // its owner has not published it yet
        const uint32_t taken = atomicAdd(&P.task_next[lo], 0u);
        if (taken + P.help_min <= total) return lo;
        if (taken >= total) atomicMax(&wc->help_lo, lo + 1);
    }
    return NONE;
}

// bmT = the transpose of the d x d bitmap bm (rows of wp words): tiles of
// 32 x 32 bits, one per warp at a time, turned by ballots.
__device__ void transpose_bitmap(const uint32_t* bm, uint32_t* bmT, uint32_t d, uint32_t wp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t x = threadIdx.x; x < d * wp; x += DBLOCK) bmT[x] = 0;
    __syncthreads();
    const uint32_t nt = (d + 31) >> 5;
    for (uint32_t t = warp; t < nt * nt; t += DW) {
        const uint32_t ti = t / nt, tj = t % nt;
        if (tj < ti) continue;  // rows only have bits above the diagonal
        const uint32_t r = ti * 32 + lane;
        const uint32_t w = r < d ? bm[(size_t)r * wp + tj] : 0u;
        uint32_t mine = 0;
        for (int b = 0; b < 32; ++b) {
            const uint32_t col = __ballot_sync(0xffffffffu, (w >> b) & 1u);
            if (lane == b) mine = col;
        }
        const uint32_t c = tj * 32 + lane;
        if (c < d) bmT[(size_t)c * wp + ti] = mine;
    }
    __syncthreads();
}

// Rows of a small root's induced sub-graph (at most 32 candidates) into
// dw.T, one word per row, and its candidates into X.scand (one warp).
__device__ __forceinline__ uint32_t small_root_rows(const CountParams& P, uint32_t u, DeepWarp& dw, const PvCtx& X) {
    const int lane = threadIdx.x & 31;
    const uint32_t b0 = P.rp[u];
    const uint32_t d = P.rp[u + 1] - b0;
    if (lane < (int)d) X.scand[lane] = P.col[b0 + lane];
    __syncwarp();
    const uint32_t last = X.scand[d - 1];
    uint32_t rb = 0, re = 0;
    if (lane < (int)d) {
        rb = __ldg(P.rp + X.scand[lane]);
        re = __ldg(P.rp + X.scand[lane] + 1);
    }
    for (uint32_t r = 0; r < d; ++r) {
        const uint32_t xb = __shfl_sync(0xffffffffu, rb, r), xe = __shfl_sync(0xffffffffu, re, r);
        uint32_t bits = 0;
        scan_row(P.col, xb, xe, last, lane, [&](uint32_t y) {
            const uint32_t pos = find_sorted(X.scand, r + 1, d, y);
            if (pos != NONE) bits |= 1u << pos;
        });
        bits = __reduce_or_sync(0xffffffffu, bits);
        if (lane == 0) dw.T[r] = bits;
    }
    __syncwarp();
    return d;
}

template <bool EC, bool PV>
__global__ void __launch_bounds__(DBLOCK) k_count_deep(const DeepParams D) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ DeepShared sh;
    __shared__ DeepSteal ss;
    const CountParams& P = D.base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wp = D.wp;
    const uint32_t D0 = (P.dcap + 31) & ~31u;
    const size_t wstride = (size_t)(D.wide_levels + 1) * wp;         // wide stack words per warp
    // layout: candidates | task prefix (EC) | per-warp areas | donated frames | hash table |
    //         bitmap | wide stacks [PV: transposed bitmap | per-warp PV areas | per-candidate gains]
    uint32_t* cand = smem;
    uint32_t* tpre = cand + D0;                                      // D0 + 32 words
    DeepWarp* dws = reinterpret_cast<DeepWarp*>(tpre + D0 + 32);
    uint32_t* qwords = reinterpret_cast<uint32_t*>(dws + DW);        // DQCAP x wp words
    uint32_t* tab = qwords + (size_t)DQCAP * wp;
    uint32_t* after_tab = tab + P.hash_words;
    uint32_t* region = P.in_smem ? after_tab : P.gscratch + (size_t)blockIdx.x * P.gscratch_words;
    uint32_t* bm = region;
    uint32_t* wide = bm + (size_t)P.dcap * wp;
    uint32_t* bmT = wide + (size_t)DW * wstride;                      // PV
    uint32_t* pv_smem = P.in_smem ? bmT + (PV ? (size_t)P.dcap * wp : 0) : after_tab;
    DeepWarpPv* pvw = reinterpret_cast<DeepWarpPv*>(pv_smem);         // PV
    unsigned long long* pvc = reinterpret_cast<unsigned long long*>(pvw + DW);  // PV: D0 + 1 entries
    DeepWarp& dw = dws[warp];
    uint32_t* stk = wide + (size_t)warp * wstride;
    PvCtx X;
    X.pvc = pvc;
    X.bmT = bmT;
    X.TT = pvw[warp].TT;
    X.pvm = pvw[warp].pvm;
    X.scand = pvw[warp].scand;
    Acc acc;
    WorkCtl* wc = reinterpret_cast<WorkCtl*>(P.ctl + 1);
    int phase = 0;
    const uint32_t k = P.k;
    for (;;) {
        if (threadIdx.x == 0) {
            sh.slot = P.n_big ? deep_next_slot(D, wc, phase) : NONE;
            sh.task = 0;
        }
        __syncthreads();
        const uint32_t s = sh.slot;
        if (s == NONE) break;
        const uint32_t u = P.roots[s];
        const uint32_t d = load_root(P.rp, P.col, u, cand);
        X.ncand = d;
        build_bitmap_hashed<DBLOCK>(P.rp, P.col, cand, d, wp, bm, tab, hash_bits_for(d));
        if (PV) {
            for (uint32_t i = threadIdx.x; i <= d; i += DBLOCK) pvc[i] = 0;
            transpose_bitmap(bm, bmT, d, wp);
        }
        // task count: VC the root's edges to its candidates, EC the edges of
        // its induced sub-graph (numbered row by row through tpre)
        if (EC) {
            if (warp == 0) {
                uint32_t carry = 0;
                for (uint32_t t0 = 0; t0 < d; t0 += 32) {
                    const uint32_t t = t0 + lane;
                    uint32_t c = 0;
                    if (t < d)
                        for (uint32_t w = (t + 1) >> 5; w < wp; ++w) c += __popc(bm[(size_t)t * wp + w]);
                    uint32_t incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    if (t < d) tpre[t] = carry + incl - c;
                    carry += __shfl_sync(0xffffffffu, incl, 31);
                }
                if (lane == 0) {
                    tpre[d] = carry;
                    sh.total = carry;
                }
            }
        } else if (threadIdx.x == 0) {
            sh.total = d;
        }
        if (threadIdx.x == 0) {
            ss.idle = 0;
            ss.active = DW;
            ss.queued = 0;
            for (int x = 0; x < DQCAP; ++x) ss.state[x] = 0;
        }
        __syncthreads();
        const uint32_t total = sh.total;
        if (threadIdx.x == 0 && P.help_min && total) atomicMax(&D.task_total[s], total);
        // EC roots have up to d^2 / 2 tasks: warps claim them in chunks
        const uint32_t chunk = EC ? max(1u, min(32u, total / (32u * DW))) : 1u;
        for (;;) {
            uint32_t t0 = 0;
            if (lane == 0) {
                t0 = timed_out(P.ctl) ? NONE
                                      : (P.help_min ? atomicAdd(&P.task_next[s], chunk) : atomicAdd(&sh.task, chunk));
            }
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            if (t0 >= total) break;
            const uint32_t t1 = min(t0 + chunk, total);
            for (uint32_t t = t0; t < t1; ++t) {
                if (!EC) {
                    // root edge u -> cand[t]: the node row t, k - 2 vertices to choose
                    const uint32_t* R = bm + (size_t)t * wp;
                    const uint32_t lo = (t + 1) >> 5;
                    const uint32_t m = warp_popc(R, lo, wp);
                    if (m + 2 >= k) {
                        const WalkStart w0{R, lo, m, k - 2, false, 0u, 0u, 0u};
                        const unsigned long long c =
                            deep_walk<PV>(D, bm, w0, stk, dw, X, acc, &ss, qwords, lane == 0 ? t : 0u, 1u);
                        if (PV && lane == 0) {
                            pv_add_at(pvc, t, d + 1, c, P.ctl, 213u);
                            pv_add_at(pvc, d, d + 1, c, P.ctl, 214u);
                        }
                    }
                } else {
                    // root triangle (u, cand[a], cand[b]), b the r-th member of row a
                    uint32_t lo_ = 0, hi_ = d;
                    while (hi_ - lo_ > 1) {
                        const uint32_t mid = (lo_ + hi_) >> 1;
                        if (tpre[mid] <= t) lo_ = mid; else hi_ = mid;
                    }
                    const uint32_t a = lo_;
                    const uint32_t* Ra = bm + (size_t)a * wp;
                    const uint32_t b = select_above(Ra, a, t - tpre[a], wp);
                    // the node row a & row b (k - 3 to choose) in the warp's first stack level;
                    // lanes may still be reading the previous task's node there
                    __syncwarp();
                    uint32_t* C = stk;
                    const uint32_t lo = (b + 1) >> 5;
                    const uint32_t* Rb = bm + (size_t)b * wp;
                    uint32_t c = 0;
                    for (uint32_t w = lane; w < wp; w += 32) {
                        const uint32_t x = w >= lo ? (Ra[w] & Rb[w]) : 0u;
                        C[w] = x;
                        c += __popc(x);
                    }
                    acc.words += (lane == 0) ? (wp - lo) : 0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                    __syncwarp();
                    if (c + 3 >= k) {
                        const WalkStart w0{C, lo, c, k - 3, false, 0u, 0u, 0u};
                        const unsigned long long n3 = deep_walk<PV>(D, bm, w0, stk + wp, dw, X, acc, &ss, qwords,
                                                                    lane == 0 ? a : (lane == 1 ? b : 0u), 2u);
                        if (PV && lane == 0) {
                            pv_add_at(pvc, a, d + 1, n3, P.ctl, 215u);
                            pv_add_at(pvc, b, d + 1, n3, P.ctl, 216u);
                            pv_add_at(pvc, d, d + 1, n3, P.ctl, 217u);
                        }
                    }
                }
            }
        }
        // out of tasks: walk frames donated by the block's busy warps
        {
            WalkStart f;
            uint32_t path_reg = 0, npath = 0;
            while (deep_steal(P.ctl, &ss, qwords, wp, stk, &f, &path_reg, &npath)) {
                const unsigned long long c =
                    deep_walk<PV>(D, bm, f, stk + wp, dw, X, acc, &ss, qwords, path_reg, npath);
                if (PV) {
                    if (lane < (int)npath) pv_add_at(pvc, path_reg, d + 1, c, P.ctl, 218u);
                    if (lane == 0) pv_add_at(pvc, d, d + 1, c, P.ctl, 219u);
                }
            }
        }
        __syncthreads();
        if (PV) {
            // this block's share of the root's per-vertex counts
            for (uint32_t i = threadIdx.x; i <= d; i += DBLOCK)
                pv_add_at(D.pv, i < d ? cand[i] : u, D.n, pvc[i], P.ctl, 220u);
            __syncthreads();
        }
    }
    __syncthreads();
    if (P.n_work > P.n_big) {
        if (!PV) {
            WarpShared* ws = reinterpret_cast<WarpShared*>(smem) + warp;
            warp_phase(P, *ws, acc);
        } else {
            // small roots: the root's candidate set is re-encoded directly
            uint32_t iter = 0;
            for (;;) {
                uint32_t i = 0;
                if (lane == 0) {
                    i = P.n_big + atomicAdd(&wc->small_cursor, 1u);
                    if ((++iter & 63u) == 0 && timed_out(P.ctl)) i = NONE;
                }
                i = __shfl_sync(0xffffffffu, i, 0);
                if (i >= P.n_work) break;
                const uint32_t u = P.roots[i];
                const uint32_t d = small_root_rows(P, u, dw, X);
                const unsigned long long e = warp_small<1, PV>(P.ctl, dw, X, d, k - 1, acc);
                const unsigned long long c = warp_sum64(e);
                for (uint32_t a = lane; a < d; a += 32) pv_add_at(D.pv, X.scand[a], D.n, X.pvm[a], P.ctl, 221u);
                if (lane == 0) pv_add_at(D.pv, u, D.n, c, P.ctl, 222u);
                __syncwarp();
            }
        }
    }
    // warp reduction (exact 128-bit), then one atomic pair per warp
    unsigned long long lo = acc.lo, hi = acc.hi, words = acc.words;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long yh = __shfl_xor_sync(0xffffffffu, hi, o);
        words += __shfl_xor_sync(0xffffffffu, words, o);
        const unsigned long long sum = lo + y;
        hi += yh + (sum < lo ? 1ull : 0ull);
        lo = sum;
    }
    if (lane == 0) {
        add_u128(&P.ctl->total_lo, &P.ctl->total_hi, lo);
        if (hi) atomicAdd(&P.ctl->total_hi, hi);
        atomicAdd(&P.ctl->words, words);
        if (P.sm_work) {
            const unsigned sm = smid();
            if (sm < SM_WORK_SLOTS) atomicAdd(&P.sm_work[sm], words);
        }
    }
}

// out[v] = pv[new_of_old[v]]: per-vertex counts in the input numbering
__global__ void k_pv_to_input(const unsigned long long* __restrict__ pv, const uint32_t* __restrict__ new_of_old,
                              uint32_t n, unsigned long long* __restrict__ out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = pv[new_of_old[v]];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static constexpr size_t DEEP_SMEM_LIMIT = 220 * 1024;

struct DeepGeometry {
    uint32_t dcap, wp, wide_levels, hash_words;
    int in_smem;
    size_t smem_bytes, gscratch_words;
};

static DeepGeometry deep_geometry(uint32_t d_max, uint32_t k, bool pv) {
    DeepGeometry g;
    g.dcap = std::max<uint32_t>(d_max, 1);
    g.wp = (((g.dcap + 31) / 32) + 3) & ~3u;
    g.wide_levels = k;  // wide levels above the re-encoded ones: fewer than k
    const size_t D0 = (g.dcap + 31) & ~31u;
    g.hash_words = g.dcap < 65535 ? hash_table_words(g.dcap) : 0;
    const size_t fixed = D0 + D0 + 32 + DW * (sizeof(DeepWarp) / 4) + (size_t)DQCAP * g.wp + g.hash_words;
    // per-vertex variant: per-warp areas and per-candidate gains stay in shared memory
    const size_t pv_fixed = pv ? DW * (sizeof(DeepWarpPv) / 4) + 2 * (D0 + 2) : 0;
    const size_t region = (size_t)g.dcap * g.wp * (pv ? 2 : 1) + (size_t)DW * (g.wide_levels + 1) * g.wp;
    const size_t warp_mode = sizeof(WarpShared) * NWARPS / 4;
    if ((fixed + pv_fixed + region) * 4 <= DEEP_SMEM_LIMIT && g.hash_words) {
        g.in_smem = 1;
        g.smem_bytes = std::max(fixed + pv_fixed + region, warp_mode) * 4;
        g.gscratch_words = 0;
    } else {
        g.in_smem = 0;
        g.smem_bytes = std::max(fixed + pv_fixed, warp_mode) * 4;
        g.gscratch_words = (region + 63) & ~(size_t)63;
    }
    return g;
}

typedef void (*DeepKernel)(const DeepParams);

static DeepKernel deep_kernel(bool ec, bool pv) {
    if (pv) return ec ? k_count_deep<true, true> : k_count_deep<false, true>;
    return ec ? k_count_deep<true, false> : k_count_deep<false, false>;
}

bool deep_supported(const kc_graph* g, uint32_t k, bool pv) {
    if (k > DEEP_MAX_K || k < (pv ? 3u : 5u)) return false;
    const DeepGeometry geo = deep_geometry(g->d_max, k, pv);
    return geo.hash_words != 0 && geo.smem_bytes <= DEEP_SMEM_LIMIT;
}

kc_status deep_plan(const kc_graph* g, uint32_t k, bool ec, bool pv, size_t* scratch_words, int* blocks_out) {
    const DeepGeometry geo = deep_geometry(g->d_max, k, pv);
    DeepKernel kern = deep_kernel(ec, pv);
    KC_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem_bytes));
    int bps = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, DBLOCK, geo.smem_bytes));
    if (bps < 1) return set_error(KC_E_UNSUPPORTED, "deep count kernel cannot be resident (smem %zu)", geo.smem_bytes);
    *blocks_out = bps * g->sm_count;
    *scratch_words = geo.gscratch_words * (size_t)(*blocks_out);
    return KC_OK;
}

kc_status deep_launch(kc_graph* g, uint32_t k, bool ec, uint32_t n_big, uint32_t n_work, uint32_t* task_next,
                      uint32_t* task_total, uint32_t* gscratch, unsigned long long* pv, Ctl* ctl, cudaStream_t s) {
    const bool pvon = pv != nullptr;
    if (pvon && k < 4) ec = false;  // an edge-centric task at k = 3 is a single clique
    const DeepGeometry geo = deep_geometry(g->d_max, k, pvon);
    DeepKernel kern = deep_kernel(ec, pvon);
    int blocks = 0;
    size_t sw = 0;
    KC_CHECK(deep_plan(g, k, ec, pvon, &sw, &blocks));
    DeepParams D;
    memset(&D, 0, sizeof(D));
    CountParams& P = D.base;
    P.rp = (const uint32_t*)g->row_ptr.ptr;
    P.col = (const uint32_t*)g->col.ptr;
    P.k = k;
    P.roots = (const uint32_t*)g->roots.ptr;
    P.n_big = n_big;
    P.n_work = n_work;
    P.task_next = task_next;
    P.help_min = 2;
    P.dcap = geo.dcap;
    P.wcap = geo.wp;
    P.in_smem = geo.in_smem;
    P.gscratch = gscratch;
    P.gscratch_words = geo.gscratch_words;
    P.hash_words = geo.hash_words;
    P.ctl = ctl;
    P.sm_work = (unsigned long long*)g->sm_work.ptr;
    D.ec = ec;
    D.wp = geo.wp;
    D.wide_levels = geo.wide_levels;
    D.task_total = task_total;
    D.pv = pv;
    D.n = g->n;
    kern<<<blocks, DBLOCK, geo.smem_bytes, s>>>(D);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status pv_to_input(const kc_graph* g, const unsigned long long* pv, uint64_t* out, cudaStream_t s) {
    if (g->n == 0) return KC_OK;
    k_pv_to_input<<<std::max(1, g->sm_count * 4), 256, 0, s>>>(pv, (const uint32_t*)g->new_of_old.ptr, g->n,
                                                               (unsigned long long*)out);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

}  // namespace kc
