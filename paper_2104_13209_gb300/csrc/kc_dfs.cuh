// Pieces of the graph-orientation traversal (Fig. 2) shared by the count
// kernels: launch parameters, exact accumulators, the time limit, root
// claiming, and warp mode for roots with at most 32 candidates.
#pragma once

#include "kc_bitmap.cuh"
#include "kc_common.cuh"

namespace kc {

static constexpr int BLOCK = 256;
static constexpr int NWARPS = BLOCK / 32;
static constexpr int SMALL_D = 32;      // warp mode handles |C| <= 32
static constexpr int WARP_DEPTH = 32;   // per-lane stack levels in warp mode
static constexpr int MAX_DEPTH = 64;    // stack levels per group in block mode
static constexpr uint32_t EC_COMPACT_MIN_K = 6;  // edge-centric: compact the edge's sub-graph from this k on

struct CountParams {
    const uint32_t* rp;        // DAG row pointers (library numbering)
    const uint32_t* col;       // DAG columns
    uint32_t k;
    const uint32_t* roots;     // library ids, decreasing out-degree
    uint32_t n_big;            // roots[0, n_big): |C| > 32 and |C| >= k - 1
    uint32_t n_work;           // roots[n_big, n_work): 32 >= |C| >= k - 1
    uint32_t* task_next;       // per big root: next unclaimed task (zeroed before launch)
    uint32_t help_min;         // join another block's root only if this many tasks are left (0 = never)
    uint32_t dcap, wcap, depth;
    int in_smem;               // bitmaps and stacks in shared memory (else per-block global scratch)
    uint32_t* gscratch;
    size_t gscratch_words;
    uint32_t hash_words;       // shared-memory words of the candidate position table (0: binary search)
    Ctl* ctl;
    unsigned long long* sm_work;  // nullable: work units per SM (SM_WORK_SLOTS entries)
};

// Extra counters of the kernel (kept right after the Ctl record).
struct WorkCtl {
    unsigned int root_cursor;   // next big root to own
    unsigned int help_lo;       // every big root below this has no unclaimed task
    unsigned int small_cursor;  // next small root
    unsigned int pad;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    const unsigned lane = threadIdx.x & 31;
    return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
}

template <int G>
__device__ __forceinline__ void group_sync(unsigned gm) {
    if (G > 1) __syncwarp(gm);
}

template <int G>
__device__ __forceinline__ uint32_t group_sum(uint32_t x, unsigned gm) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(gm, x, o);
    return x;
}

struct Acc {
    unsigned long long lo = 0, hi = 0, words = 0;
    __device__ __forceinline__ void add(unsigned long long x) {
        lo += x;
        hi += (lo < x) ? 1ull : 0ull;
    }
};

// True once %globaltimer has passed the launch's deadline (every warp reads
// the same clock, so no flag needs to be polled: the check costs one cached
// load and a special-register read, cheap enough for the inner loops).
__device__ __forceinline__ bool timed_out(const Ctl* c) {
    if (c->deadline == 0) return false;
    if (globaltimer_ns() > c->deadline) {
        atomicOr((unsigned*)&c->flags, (unsigned)KC_FLAG_TIMEOUT);
        return true;
    }
    return false;
}

struct BlockShared {
    uint32_t slot;
    uint32_t task;      // next unclaimed task of a root no other block can join
    uint32_t edge;
    uint32_t sub_next;
    uint32_t sub_d;
};


// Candidate list of root u into cand[]; returns d.
__device__ __forceinline__ uint32_t load_root(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                              uint32_t u, uint32_t* cand) {
    const uint32_t b = rp[u], d = rp[u + 1] - b;
    for (uint32_t i = threadIdx.x; i < d; i += BLOCK) cand[i] = col[b + i];
    __syncthreads();
    return d;
}

// Pick the next big root for this block: own a new one while any is left,
// then join roots in which other blocks still have unclaimed tasks.
static __device__ uint32_t next_big_slot(const CountParams& P, WorkCtl* wc, int& phase) {
    if (timed_out(P.ctl)) return NONE;
    if (phase == 0) {
        uint32_t s = atomicAdd(&wc->root_cursor, 1u);
        if (s < P.n_big) return s;
        phase = 1;
    }
    if (P.help_min == 0) return NONE;
    uint32_t lo = atomicAdd(&wc->help_lo, 0u);
    for (uint32_t probes = 0; lo < P.n_big && probes < 4096; ++lo, ++probes) {
        const uint32_t u = P.roots[lo];
        const uint32_t d = P.rp[u + 1] - P.rp[u];
        const uint32_t taken = atomicAdd(&P.task_next[lo], 0u);
        if (taken + P.help_min <= d) return lo;
        if (taken >= d) atomicMax(&wc->help_lo, lo + 1);
    }
    return NONE;
}

// ---------------------------------------------------------------------------
// Warp mode (|C| <= 32): rows are single words
// ---------------------------------------------------------------------------
struct WarpShared {
    uint32_t cand[32];
    uint32_t filt[32];     // candidate filter (1,024 bits: one word per bank, so lookups never conflict)
    uint32_t row[32];
    uint32_t pre[32];      // exclusive prefix of the rows' popcounts (level-3 task numbering)
    uint32_t next;         // next unclaimed level-3 task
    uint32_t stk[WARP_DEPTH * 32];
};

// sum over j in c of popc(c & row_j)
__device__ __forceinline__ uint32_t edge_count1(uint32_t c, const uint32_t* row) {
    uint32_t s = 0;
    while (c) {
        uint32_t j = __ffs(c) - 1;
        c &= c - 1;
        s += __popc(c & row[j]);
    }
    return s;
}

// number of rem0-subsets of J (ascending choice) that are cliques, rem0 >= 3
static __device__ uint64_t lane_walk(const CountParams& P, uint32_t J0, uint32_t rem0, const uint32_t* row, uint32_t* stk,
                              unsigned long long& words) {
    const int lane = threadIdx.x & 31;
    uint64_t acc = 0;
    int l = 0;
    stk[lane] = J0;
    uint32_t steps = 0;
    for (;;) {
        uint32_t J = stk[l * 32 + lane];
        const uint32_t rem = rem0 - l;
        if ((uint32_t)__popc(J) < rem) {
            if (l == 0) break;
            --l;
            continue;
        }
        if ((++steps & 1023u) == 0 && timed_out(P.ctl)) break;
        uint32_t v = __ffs(J) - 1;
        J &= J - 1;
        stk[l * 32 + lane] = J;
        uint32_t c = J & row[v];
        ++words;
        const uint32_t need = rem - 1;
        if ((uint32_t)__popc(c) < need) continue;
        if (need == 2) {
            acc += edge_count1(c, row);
            words += __popc(c);
            continue;
        }
        ++l;
        stk[l * 32 + lane] = c;
    }
    return acc;
}

// One small root u (at most 32 candidates) by one warp: one-word rows built
// cooperatively, then lane i walks the subtree below the root edge
// u -> cand[i].  rp / col: the root's DAG; k: its query's clique size.
static __device__ void warp_root(const CountParams& P, const uint32_t* __restrict__ rp, const uint32_t* __restrict__ col,
                          uint32_t k, uint32_t u, WarpShared& ws, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const uint32_t rem0 = k - 2;  // below the root edge u -> cand[lane]
    const uint32_t b = rp[u];
    const uint32_t d = rp[u + 1] - b;
    constexpr uint32_t FBITS = 10;  // 1,024 filter bits for at most 32 candidates
    uint32_t cu = 0;
    if (lane < (int)d) {
        cu = col[b + lane];
        ws.cand[lane] = cu;
    }
    ws.filt[lane] = 0;
    __syncwarp();
    if (lane < (int)d) {
        const uint32_t hf = hash_slot(cu, FBITS);
        atomicOr(&ws.filt[hf >> 5], 1u << (hf & 31));
    }
    __syncwarp();
    // rows, one per candidate, built cooperatively (lanes over N+(cand[r]));
    // lane r holds the bounds of row r, loaded together
    const uint32_t last = ws.cand[d - 1];
    uint32_t rb = 0, re = 0;
    if (lane < (int)d) {
        rb = __ldg(rp + cu);
        re = __ldg(rp + cu + 1);
    }
    for (uint32_t r = 0; r < d; ++r) {
        const uint32_t xb = __shfl_sync(0xffffffffu, rb, r), xe = __shfl_sync(0xffffffffu, re, r);
        uint32_t bits = 0;
        scan_row_filtered(col, xb, xe, last, lane, ws.filt, FBITS, [&](uint32_t y) {
            const uint32_t pos = find_sorted(ws.cand, r + 1, d, y);
            if (pos != NONE) bits |= 1u << pos;
        });
        bits = __reduce_or_sync(0xffffffffu, bits);
        if (lane == 0) ws.row[r] = bits;
    }
    __syncwarp();
    if (rem0 <= 2) {
        // lane i counts below the root edge u -> cand[i] (one or two levels)
        if (lane < (int)d) {
            const uint32_t R = ws.row[lane];
            uint64_t c = 0;
            if (rem0 == 1) {
                c = __popc(R);
            } else {
                c = edge_count1(R, ws.row);
                acc.words += __popc(R);
            }
            acc.add(c);
        }
        __syncwarp();
        return;
    }
    // deeper trees: the level-3 subtrees (u, cand[i], cand[j]), j in row i,
    // numbered row by row, are claimed one at a time by the lanes, so that a
    // dense root's work spreads over the warp
    const uint32_t cnt = lane < (int)d ? __popc(ws.row[lane]) : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    ws.pre[lane] = incl - cnt;
    const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) ws.next = 0;
    __syncwarp();
    const uint32_t rem1 = rem0 - 1;
    uint64_t c = 0;
    for (;;) {
        const uint32_t t = atomicAdd(&ws.next, 1u);
        if (t >= T) break;
        uint32_t lo = 0, hi = d;  // the row i with pre[i] <= t < pre[i] + popc(row i)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (ws.pre[mid] <= t) lo = mid; else hi = mid;
        }
        const uint32_t Ri = ws.row[lo];
        const uint32_t j = __fns(Ri, 0, (int)(t - ws.pre[lo]) + 1);
        const uint32_t J = Ri & ws.row[j];
        ++acc.words;
        if ((uint32_t)__popc(J) < rem1) continue;
        if (rem1 == 2) {
            c += edge_count1(J, ws.row);
            acc.words += __popc(J);
        } else {
            c += lane_walk(P, J, rem1, ws.row, ws.stk, acc.words);
        }
    }
    acc.add(c);
    __syncwarp();
}

// Small roots of a single-graph launch, one per warp from a global cursor.
static __device__ void warp_phase(const CountParams& P, WarpShared& ws, Acc& acc) {
    WorkCtl* wc = reinterpret_cast<WorkCtl*>(P.ctl + 1);
    const int lane = threadIdx.x & 31;
    uint32_t iter = 0;
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) {
            i = P.n_big + atomicAdd(&wc->small_cursor, 1u);
            if ((++iter & 63u) == 0 && timed_out(P.ctl)) i = NONE;
        }
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= P.n_work) break;
        warp_root(P, P.rp, P.col, P.k, P.roots[i], ws, acc);
    }
}

}  // namespace kc
