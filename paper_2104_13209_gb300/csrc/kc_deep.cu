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
};

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

// Edges of the sub-graph induced by J (rows T, nw words each).
template <int NW>
__device__ __forceinline__ unsigned long long lane_edges(Mask<NW> J, const uint32_t* T, unsigned long long& words) {
    unsigned long long s = 0;
    for (;;) {
        const uint32_t v = mask_pop<NW>(J);
        if (v == NONE) break;
        s += mask_popc<NW>(mask_and<NW>(J, T + (size_t)v * NW));
        words += NW;
    }
    return s;
}

// rem-cliques of the sub-graph induced by J0 (rem >= 3), one lane alone.
template <int NW>
__device__ unsigned long long lane_walk_nw(const Ctl* ctl, Mask<NW> J0, uint32_t rem0, const uint32_t* T,
                                           unsigned long long& words) {
    Mask<NW> stk[LANE_DEPTH];
    unsigned long long acc = 0;
    int l = 0;
    stk[0] = J0;
    uint32_t steps = 0;
    for (;;) {
        Mask<NW>& J = stk[l];
        const uint32_t rem = rem0 - l;
        if (mask_popc<NW>(J) < rem) {
            if (l == 0) break;
            --l;
            continue;
        }
        if ((++steps & 65535u) == 0 && timed_out(ctl)) break;
        const uint32_t v = mask_pop<NW>(J);
        const Mask<NW> C = mask_and<NW>(J, T + (size_t)v * NW);
        words += NW;
        const uint32_t c = mask_popc<NW>(C);
        const uint32_t need = rem - 1;
        if (c < need) continue;
        if (need == 1) {
            acc += c;
        } else if (need == 2) {
            acc += lane_edges<NW>(C, T, words);
        } else {
            stk[++l] = C;
        }
    }
    return acc;
}

// rem-cliques (rem >= 2) of the re-encoded sub-graph on m vertices held in
// dw.T, by the 32 lanes of the warp.  rem == 2: lanes take rows; rem == 3:
// lanes take rows and count each row's edges; rem == 4: lanes claim rows and
// count the edges below each of their edges; rem >= 5: lanes claim the edges
// (a, b) of the sub-graph one at a time and walk below a & b.
template <int NW>
__device__ void warp_small(const Ctl* ctl, DeepWarp& dw, uint32_t m, uint32_t rem, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const uint32_t* T = dw.T;
    if (rem <= 3) {
        unsigned long long s = 0;
        for (uint32_t a = lane; a < m; a += 32) {
            Mask<NW> R;
#pragma unroll
            for (int i = 0; i < NW; ++i) R.w[i] = T[a * NW + i];
            if (rem == 2) {
                s += mask_popc<NW>(R);
                acc.words += NW;
            } else {
                s += lane_edges<NW>(R, T, acc.words);
            }
        }
        acc.add(s);
        __syncwarp();
        return;
    }
    if (rem == 4) {
        // lanes claim rows; below each edge (a, b) of a row, count the edges of a & b
        if (lane == 0) dw.next = 0;
        __syncwarp();
        unsigned long long s = 0;
        for (;;) {
            const uint32_t a = atomicAdd(&dw.next, 1u);
            if (a >= m) break;
            Mask<NW> R;
#pragma unroll
            for (int i = 0; i < NW; ++i) R.w[i] = T[a * NW + i];
            Mask<NW> B = R;
            for (;;) {
                const uint32_t b = mask_pop<NW>(B);
                if (b == NONE) break;
                const Mask<NW> J = mask_and<NW>(R, T + (size_t)b * NW);
                acc.words += NW;
                if (mask_popc<NW>(J) >= 2) s += lane_edges<NW>(J, T, acc.words);
            }
        }
        acc.add(s);
        __syncwarp();
        return;
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
    unsigned long long s = 0;
    for (;;) {
        const uint32_t t = atomicAdd(&dw.next, 1u);
        if (t >= total) break;
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
        if (rem2 == 1) s += c;
        else if (rem2 == 2) s += lane_edges<NW>(J, T, acc.words);
        else s += lane_walk_nw<NW>(ctl, J, rem2, T, acc.words);
    }
    acc.add(s);
    __syncwarp();
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

// Re-encode the sub-graph induced by L (m <= CMAX members) into dw.T with NW
// words per row: bit b of row a iff pos[b] is in row pos[a] of bm.
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
// the members (positions from a word prefix), each sums popc(L & row_j) from
// j's word on.
__device__ __forceinline__ unsigned long long wide_edges(const uint32_t* L, const uint32_t* bm, uint32_t wp,
                                                         uint32_t lo, unsigned long long& words) {
    const int lane = threadIdx.x & 31;
    unsigned long long s = 0;
    // lanes take words of L round-robin and the members in them
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

// The node (L, rem) of the root's tree: L has m members (m >= rem), its
// words below lo are zero.  stk: the warp's wide stack (levels x wp words).
__device__ void deep_node(const DeepParams& D, const uint32_t* bm, const uint32_t* L0, uint32_t lo0, uint32_t m0,
                          uint32_t rem0, uint32_t* stk, DeepWarp& dw, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const uint32_t wp = D.wp;
    const Ctl* ctl = D.base.ctl;
    // explicit stack of wide levels: list, cursor, members left above the cursor
    uint32_t cur[LANE_DEPTH], left[LANE_DEPTH];
    const uint32_t* Ls[LANE_DEPTH];
    int l = -1;
    const uint32_t* L = L0;
    uint32_t lo = lo0, m = m0, rem = rem0;
    uint32_t steps = 0;
    for (;;) {
        // analyse the node (L, lo, m, rem)
        bool descend = false;
        if (rem == 1) {
            if (lane == 0) acc.add(m);
        } else if (rem == 2) {
            acc.add(wide_edges(L, bm, wp, lo, acc.words));
        } else if (m <= CMAX) {
            list_members(L, wp, dw);
            if (m <= 32) {
                reencode<1>(bm, wp, m, dw);
                warp_small<1>(ctl, dw, m, rem, acc);
            } else if (m <= 64) {
                reencode<2>(bm, wp, m, dw);
                warp_small<2>(ctl, dw, m, rem, acc);
            } else {
                reencode<4>(bm, wp, m, dw);
                warp_small<4>(ctl, dw, m, rem, acc);
            }
        } else if (l + 1 < (int)D.wide_levels && l + 1 < LANE_DEPTH) {
            descend = true;
        } else if (lane == 0) {
            atomicOr((unsigned*)&ctl->flags, (unsigned)KC_FLAG_INTERNAL);  // cannot happen: depth < k
        }
        if (descend) {
            ++l;
            Ls[l] = L;
            cur[l] = lo * 32 - 1;  // before the first member (NONE when lo == 0; next_bit starts at cur + 1)
            left[l] = m;
        }
        // next child of the deepest wide level that still has one
        for (;;) {
            if (l < 0) return;
            const uint32_t r = rem0 - (uint32_t)l;  // rem of level l's node
            if (left[l] < r) {
                --l;
                continue;
            }
            if ((++steps & 1023u) == 0) {
                int to = lane == 0 ? (int)timed_out(ctl) : 0;
                if (__shfl_sync(0xffffffffu, to, 0)) return;
            }
            const uint32_t v = next_bit(Ls[l], cur[l] + 1, wp - 1);  // cur = NONE wraps to 0
            if (v == NONE) {
                --l;
                continue;
            }
            cur[l] = v;
            --left[l];
            uint32_t* C = stk + (size_t)l * wp;
            const uint32_t clo = (v + 1) >> 5;
            const uint32_t* rv = bm + (size_t)v * wp;
            __syncwarp();
            uint32_t c = 0;
            for (uint32_t w = lane; w < wp; w += 32) {
                const uint32_t x = w >= clo ? (Ls[l][w] & rv[w]) : 0u;
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

template <bool EC>
__global__ void __launch_bounds__(DBLOCK) k_count_deep(const DeepParams D) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ DeepShared sh;
    const CountParams& P = D.base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wp = D.wp;
    const uint32_t D0 = (P.dcap + 31) & ~31u;
    // layout: candidates | task prefix (EC) | per-warp areas | hash table | bitmap | wide stacks
    uint32_t* cand = smem;
    uint32_t* tpre = cand + D0;                                      // D0 + 32 words
    DeepWarp* dws = reinterpret_cast<DeepWarp*>(tpre + D0 + 32);
    uint16_t* tab = reinterpret_cast<uint16_t*>(dws + DW);
    uint32_t* after_tab = reinterpret_cast<uint32_t*>(tab) + P.hash_words;
    uint32_t* bm;
    uint32_t* wide;
    if (P.in_smem) {
        bm = after_tab;
        wide = bm + (size_t)P.dcap * wp;
    } else {
        bm = P.gscratch + (size_t)blockIdx.x * P.gscratch_words;
        wide = bm + (size_t)P.dcap * wp;
    }
    DeepWarp& dw = dws[warp];
    uint32_t* stk = wide + (size_t)warp * D.wide_levels * wp;
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
        build_bitmap_hashed<DBLOCK>(P.rp, P.col, cand, d, wp, bm, tab, hash_bits_for(d));
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
                if (m + 2 >= k) deep_node(D, bm, R, lo, m, k - 2, stk, dw, acc);
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
                // the node row a & row b (k - 3 to choose) in the warp's first stack level
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
                if (c + 3 >= k) deep_node(D, bm, C, lo, c, k - 3, stk + wp, dw, acc);
            }
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (P.n_work > P.n_big) {
        WarpShared* ws = reinterpret_cast<WarpShared*>(smem) + warp;
        warp_phase(P, *ws, acc);
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
    }
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

static DeepGeometry deep_geometry(uint32_t d_max, uint32_t k, bool ec) {
    DeepGeometry g;
    g.dcap = std::max<uint32_t>(d_max, 1);
    g.wp = (((g.dcap + 31) / 32) + 3) & ~3u;
    g.wide_levels = k;  // wide levels above the re-encoded ones: fewer than k
    const size_t D0 = (g.dcap + 31) & ~31u;
    uint32_t b = 6;
    while ((1u << b) < 4 * g.dcap) ++b;
    g.hash_words = g.dcap < 65535 ? (1u << b) / 2 : 0;
    const size_t fixed = D0 + D0 + 32 + DW * (sizeof(DeepWarp) / 4) + g.hash_words;
    const size_t region = (size_t)g.dcap * g.wp + (size_t)DW * g.wide_levels * g.wp;
    const size_t warp_mode = sizeof(WarpShared) * NWARPS / 4;
    if ((fixed + region) * 4 <= DEEP_SMEM_LIMIT && g.hash_words) {
        g.in_smem = 1;
        g.smem_bytes = std::max(fixed + region, warp_mode) * 4;
        g.gscratch_words = 0;
    } else {
        g.in_smem = 0;
        g.smem_bytes = std::max(fixed, warp_mode) * 4;
        g.gscratch_words = (region + 63) & ~(size_t)63;
    }
    (void)ec;
    return g;
}

typedef void (*DeepKernel)(const DeepParams);

bool deep_supported(const kc_graph* g, uint32_t k) {
    if (k < 5 || k > DEEP_MAX_K) return false;
    const DeepGeometry geo = deep_geometry(g->d_max, k, false);
    return geo.hash_words != 0;
}

kc_status deep_plan(const kc_graph* g, uint32_t k, bool ec, size_t* scratch_words, int* blocks_out) {
    const DeepGeometry geo = deep_geometry(g->d_max, k, ec);
    DeepKernel kern = ec ? k_count_deep<true> : k_count_deep<false>;
    KC_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem_bytes));
    int bps = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, DBLOCK, geo.smem_bytes));
    if (bps < 1) return set_error(KC_E_UNSUPPORTED, "deep count kernel cannot be resident (smem %zu)", geo.smem_bytes);
    *blocks_out = bps * g->sm_count;
    *scratch_words = geo.gscratch_words * (size_t)(*blocks_out);
    return KC_OK;
}

kc_status deep_launch(kc_graph* g, uint32_t k, bool ec, uint32_t n_big, uint32_t n_work, uint32_t* task_next,
                      uint32_t* task_total, uint32_t* gscratch, Ctl* ctl, cudaStream_t s) {
    const DeepGeometry geo = deep_geometry(g->d_max, k, ec);
    DeepKernel kern = ec ? k_count_deep<true> : k_count_deep<false>;
    int blocks = 0;
    size_t sw = 0;
    KC_CHECK(deep_plan(g, k, ec, &sw, &blocks));
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
    D.ec = ec;
    D.wp = geo.wp;
    D.wide_levels = geo.wide_levels;
    D.task_total = task_total;
    kern<<<blocks, DBLOCK, geo.smem_bytes, s>>>(D);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

}  // namespace kc
