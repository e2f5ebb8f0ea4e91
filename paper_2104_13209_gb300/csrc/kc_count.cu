// Graph-orientation k-clique counting (Fig. 2; Sections 2.4, 3.2-3.6).
//
// A root r (every vertex with out-degree >= k-1, taken in decreasing
// out-degree order so the largest trees start first) has candidate set
// C = N+(r), listed in ascending library id.  Its induced sub-graph is binary
// encoded (Section 3.4): row i has bit j set iff C[j] is an out-neighbour of
// C[i].  The library numbering is a topological order, so row i only has
// bits j > i.
//
// Below a tree node with candidate list I (a bitmap) and `rem` vertices still
// to choose, the explicit-stack DFS (Section 3.3) does:
//   rem == 1:  count += popc(I)
//   rem == 2:  count += sum over j in I of popc(I & row_j)   (the last two levels)
//   rem >= 3:  for each v in I (ascending): I' = I & row_v, descend with rem - 1,
//              skipping v once fewer than rem bits of I remain, and skipping
//              I' when popc(I') < rem - 1 (no clique of the size can follow).
//
// Work distribution (Section 3.2):
//   vertex-centric (VC): level-2 subtrees (the edges r -> C[i]) are the tasks;
//     groups of G threads (Section 3.5) claim them from a per-root counter in
//     global memory, so several blocks can share one large root;
//   edge-centric (EC): a block takes one root edge r -> C[i] at a time, extracts
//     the compacted sub-graph induced by C ∩ N+(C[i]) (the common
//     out-neighbours of the edge's endpoints) from the root's bitmap, and its
//     groups claim the level-3 subtrees of that edge.  Blocks share a root's
//     edges through the same per-root counter.
//   Roots with |C| <= 32 run in warp mode: one warp per root, every row is one
//     32-bit word and every lane walks the subtree of one root edge.
// Blocks are persistent (Section 3.6).  Counts are summed per thread, per
// warp, then into an exact 128-bit total with carry detection.
#include <algorithm>
#include <mutex>

#include "kc_dfs.cuh"

namespace kc {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Block mode
// ---------------------------------------------------------------------------
// sum over j in I of popc(I & row_j), words [lo, hi] (the last level of the
// traversal: every edge of the sub-graph induced by I closes a clique).
// Thread gl of the group takes the words lo + gl, lo + gl + G, ... of I and,
// for each member j found there, sums the row words from j's own word on by
// itself (rows are upper triangular).  Most lists at this level are sparse,
// so splitting the scan of I beats stepping through its members together.
template <int G>
__device__ __forceinline__ void edge_count(const uint32_t* I, const uint32_t* bm, uint32_t W, uint32_t lo, uint32_t hi,
                                           unsigned gl, Acc& acc) {
    for (uint32_t w = lo + gl; w <= hi; w += G) {
        uint32_t bits = I[w];
        while (bits) {
            uint32_t j = (w << 5) + (__ffs(bits) - 1);
            bits &= bits - 1;
            const uint32_t* rj = bm + (size_t)j * W;
            uint32_t s = 0;
            for (uint32_t x = w; x <= hi; ++x) s += __popc(I[x] & rj[x]);
            acc.add(s);
            acc.words += hi - w + 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Work stealing between the groups of a block.  A frame is one level of a
// walk: a candidate list L (W words), the candidates still to branch on
// (bits of L above `cursor` and below `end`), the number of vertices still
// to choose (`rem`) and the number of bits of L above the cursor (`cnt`, for
// the size bound).  A busy group that sees idle groups donates the upper half
// of the remaining candidates of its shallowest frame through a small queue
// in shared memory; the donor stops its own iteration below the split.
// ---------------------------------------------------------------------------
static constexpr int QCAP = 16;
// A waiting group gives up after IDLE_NS (%globaltimer) and leaves the
// pool; the groups that still hold work finish it themselves, so leaving is
// always safe (the count stays exact).
static constexpr unsigned long long IDLE_NS = 2000000000ull;

struct StealShared {
    unsigned idle;        // groups waiting for work (or trying to take some)
    unsigned active;      // groups still in the session
    unsigned queued;      // frames ready in the queue
    unsigned state[QCAP]; // 0 empty, 1 being written, 2 ready, 3 being read
    unsigned meta[QCAP][4];
};

__device__ __forceinline__ unsigned vld(const unsigned* p) { return *(const volatile unsigned*)p; }

// bits of L strictly between a and b (positions), summed over the group
template <int G>
__device__ __forceinline__ uint32_t range_popc(const uint32_t* L, uint32_t a, uint32_t b, uint32_t W, unsigned gl,
                                               unsigned gm) {
    uint32_t c = 0;
    const uint32_t lo = a + 1;
    if (lo < b) {
        const uint32_t w0 = lo >> 5, w1 = min((b - 1) >> 5, W - 1);
        for (uint32_t w = w0 + gl; w <= w1; w += G) {
            uint32_t x = L[w];
            if (w == w0) x &= 0xFFFFFFFFu << (lo & 31);
            if (w == ((b - 1) >> 5)) x &= 0xFFFFFFFFu >> (31 - ((b - 1) & 31));
            c += __popc(x);
        }
    }
    return group_sum<G>(c, gm);
}

// The subtree walk from a frame (L0, cursor0, end0, cnt0, rem0 >= 3) by the
// G threads of one group.  stk: the group's child lists (depth x W).
template <int G>
__device__ void walk_frame(const CountParams& P, const uint32_t* bm, uint32_t W, const uint32_t* L0, uint32_t cur0,
                           uint32_t end0, uint32_t cnt0, uint32_t rem0, uint32_t* stk, Acc& acc, StealShared* ss,
                           uint32_t* qwords, uint32_t qstride) {
    const unsigned gm = group_mask<G>();
    const unsigned gl = threadIdx.x & (G - 1);
    const unsigned leader = (threadIdx.x & 31) & ~(unsigned)(G - 1);
    const uint32_t hiw = W - 1;
    uint32_t cur[MAX_DEPTH + 2];
    uint32_t idx[MAX_DEPTH + 2];
    uint32_t cnt[MAX_DEPTH + 2];
    uint32_t endl[MAX_DEPTH + 2];
    int l = 0;
    cur[0] = cur0;
    idx[0] = 0;
    cnt[0] = cnt0;
    endl[0] = end0;
    uint32_t steps = 0;
    for (;;) {
        if ((++steps & 63u) == 0) {
            if ((steps & 4095u) == 0) {
                int to = gl == 0 ? (int)timed_out(P.ctl) : 0;
                if (__shfl_sync(gm, to, leader)) break;
            }
            // donate half of the shallowest frame that still has >= 2 candidates
            int want = 0;
            if (gl == 0) want = vld(&ss->idle) > 0 && vld(&ss->queued) < QCAP;
            if (__shfl_sync(gm, want, leader)) {
                for (int lv = 0; lv <= l; ++lv) {
                    const uint32_t* Lv = (lv == 0) ? L0 : stk + (size_t)(lv - 1) * W;
                    const uint32_t r = range_popc<G>(Lv, cur[lv], endl[lv], W, gl, gm);
                    if (r < 2) continue;
                    uint32_t q = NONE, split = NONE;
                    if (gl == 0) {
                        split = select_above(Lv, cur[lv], r / 2, W);
                        for (uint32_t x = 0; x < QCAP; ++x)
                            if (vld(&ss->state[x]) == 0 && atomicCAS(&ss->state[x], 0u, 1u) == 0u) {
                                q = x;
                                break;
                            }
                    }
                    q = __shfl_sync(gm, q, leader);
                    split = __shfl_sync(gm, split, leader);
                    if (q == NONE || split == NONE) break;
                    uint32_t* dst = qwords + (size_t)q * qstride;
                    for (uint32_t w = gl; w < W; w += G) dst[w] = Lv[w];
                    const uint32_t tc = range_popc<G>(Lv, split - 1, 0xFFFFFFFFu, W, gl, gm);
                    if (gl == 0) {
                        ss->meta[q][0] = split - 1;
                        ss->meta[q][1] = endl[lv];
                        ss->meta[q][2] = rem0 - lv;
                        ss->meta[q][3] = tc;
                    }
                    group_sync<G>(gm);
                    if (gl == 0) {
                        __threadfence_block();
                        atomicExch(&ss->state[q], 2u);
                        atomicAdd(&ss->queued, 1u);
                    }
                    endl[lv] = split;
                    break;
                }
            }
        }
        const uint32_t* L = (l == 0) ? L0 : stk + (size_t)(l - 1) * W;
        const uint32_t rem = rem0 - l;
        uint32_t v = (cnt[l] - idx[l] < rem) ? NONE : next_bit(L, cur[l] + 1, hiw);
        if (v != NONE && v >= endl[l]) v = NONE;
        if (v == NONE) {
            if (l == 0) break;
            --l;
            continue;
        }
        idx[l]++;
        cur[l] = v;
        const uint32_t* rv = bm + (size_t)v * W;
        uint32_t* C = stk + (size_t)l * W;
        const uint32_t lo = (v + 1) >> 5;
        group_sync<G>(gm);  // every reader of the previous sibling's list is done
        uint32_t c = 0;
        for (uint32_t w = lo + gl; w <= hiw; w += G) {
            uint32_t x = L[w] & rv[w];
            C[w] = x;
            c += __popc(x);
        }
        if (gl == 0) acc.words += hiw - lo + 1;
        c = group_sum<G>(c, gm);
        group_sync<G>(gm);
        const uint32_t need = rem - 1;
        if (c < need) continue;
        if (need == 2) {
            edge_count<G>(C, bm, W, lo, hiw, gl, acc);
            continue;
        }
        ++l;
        cur[l] = v;
        idx[l] = 0;
        cnt[l] = c;
        endl[l] = 0xFFFFFFFFu;
    }
}

// The subtree below task vertex t of bitmap bm: choose rem0 more vertices
// from row t.
template <int G>
__device__ void walk_task(const CountParams& P, const uint32_t* bm, uint32_t W, uint32_t t, uint32_t rem0,
                          uint32_t* stk, Acc& acc, StealShared* ss, uint32_t* qwords, uint32_t qstride) {
    const unsigned gm = group_mask<G>();
    const unsigned gl = threadIdx.x & (G - 1);
    const uint32_t hiw = W - 1;
    const uint32_t* R = bm + (size_t)t * W;
    const uint32_t lo0 = (t + 1) >> 5;
    if (rem0 == 0) {
        if (gl == 0) acc.add(1);
        return;
    }
    if (rem0 == 1) {
        uint32_t s = 0;
        for (uint32_t w = lo0 + gl; w <= hiw; w += G) s += __popc(R[w]);
        acc.add(s);
        return;
    }
    if (rem0 == 2) {
        edge_count<G>(R, bm, W, lo0, hiw, gl, acc);
        return;
    }
    uint32_t c0 = 0;
    for (uint32_t w = lo0 + gl; w <= hiw; w += G) c0 += __popc(R[w]);
    c0 = group_sum<G>(c0, gm);
    if (c0 < rem0) return;
    walk_frame<G>(P, bm, W, R, t, 0xFFFFFFFFu, c0, rem0, stk, acc, ss, qwords, qstride);
}

// A group out of tasks: take a donated frame, or wait until one appears or
// every group of the session is idle.  Returns true when a frame was copied
// to own (W words) with its meta in m; false when the session is over for
// this group.
template <int G>
__device__ bool steal_or_finish(const CountParams& P, StealShared* ss, uint32_t* qwords, uint32_t qstride,
                                uint32_t W, uint32_t* own, uint32_t* m) {
    const unsigned gm = group_mask<G>();
    const unsigned gl = threadIdx.x & (G - 1);
    const unsigned leader = (threadIdx.x & 31) & ~(unsigned)(G - 1);
    uint32_t q = NONE;
    int done = 0;
    if (gl == 0) {
        atomicAdd(&ss->idle, 1u);
        uint32_t it = 0;
        const unsigned long long t0 = globaltimer_ns();
        for (;; ++it) {
            if ((it & 255u) == 255u && globaltimer_ns() - t0 > IDLE_NS) break;
            if (vld(&ss->queued) > 0) {
                atomicSub(&ss->idle, 1u);  // trying to take work: no longer idle
                for (uint32_t x = 0; x < QCAP; ++x)
                    if (vld(&ss->state[x]) == 2u && atomicCAS(&ss->state[x], 2u, 3u) == 2u) {
                        q = x;
                        break;
                    }
                if (q != NONE) {
                    atomicSub(&ss->queued, 1u);
                    break;
                }
                atomicAdd(&ss->idle, 1u);
            }
            if (vld(&ss->idle) == vld(&ss->active) && vld(&ss->queued) == 0) {
                done = 1;
                break;
            }
            if ((it & 1023u) == 1023u && timed_out(P.ctl)) {
                atomicSub(&ss->idle, 1u);
                atomicSub(&ss->active, 1u);
                done = 1;
                break;
            }
            __nanosleep(256);
        }
        if (q == NONE && !done) {  // waited long enough: leave the pool (the donors finish their own work)
            atomicSub(&ss->idle, 1u);
            atomicSub(&ss->active, 1u);
            done = 1;
        }
    }
    q = __shfl_sync(gm, q, leader);
    if (q == NONE) return false;
    __threadfence_block();
    const uint32_t* src = qwords + (size_t)q * qstride;
    for (uint32_t w = gl; w < W; w += G) own[w] = src[w];
    if (gl == 0)
        for (int x = 0; x < 4; ++x) m[x] = ss->meta[q][x];
    group_sync<G>(gm);
    if (gl == 0) atomicExch(&ss->state[q], 0u);
    return true;
}

// One big root u (candidate list N+(u) with more than 32 members) by the
// whole block: the bitmap of its induced sub-graph, then the level-2 (VC) or
// root-edge (EC) subtrees claimed by the groups, then stealing until every
// group is idle.  rp / col: the DAG the root belongs to; k: the clique size
// of its query; s: the root's slot in P.task_next (used only when other
// blocks may join, P.help_min != 0).  The caller sets sh.task = 0 and
// synchronises the block before the call.
template <int G, bool EC>
__device__ void block_root(const CountParams& P, const uint32_t* __restrict__ rp, const uint32_t* __restrict__ col,
                           uint32_t k, uint32_t s, uint32_t u, uint32_t* smem, BlockShared& sh, StealShared& ss,
                           Acc& acc) {
    const uint32_t W0 = P.wcap;
    const uint32_t D0 = (P.dcap + 31) & ~31u;
    uint32_t* cand = smem;
    uint32_t* region = P.in_smem ? smem + D0 : P.gscratch + (size_t)blockIdx.x * P.gscratch_words;
    uint32_t* bm = region;                                    // dcap x W0
    // edge-centric split: the edge's induced sub-graph is compacted only when
    // the tree below it is deep enough to repay the compaction
    const bool compact = EC && k >= EC_COMPACT_MIN_K;
    uint32_t* sub = bm + (size_t)P.dcap * W0;                      // compaction: dcap x W0
    uint32_t* subidx = sub + (compact ? (size_t)P.dcap * W0 : 0);  // compaction: D0 member positions
    uint32_t* wpre = subidx + (compact ? D0 : 0);                  // compaction: W0 + 1 prefix popcounts
    uint32_t* qwords = wpre + (compact ? W0 + 32 : 0);             // QCAP x W0 donated lists
    uint32_t* stk_base = qwords + (size_t)QCAP * W0;
    uint32_t* own = stk_base + (size_t)(threadIdx.x / G) * (P.depth + 1) * W0;  // a taken frame's list
    uint32_t* stk = own + W0;                                                    // child lists
    uint32_t* tab = stk_base + (size_t)(BLOCK / G) * (P.depth + 1) * W0;
    const unsigned gm = group_mask<G>();
    const unsigned gl = threadIdx.x & (G - 1);
    const unsigned leader = (threadIdx.x & 31) & ~(unsigned)(G - 1);
    __shared__ uint32_t s_meta[BLOCK][4];  // a taken frame's meta, one row per group leader
    uint32_t* m = s_meta[threadIdx.x / G * G];
    {
        const uint32_t d = load_root(rp, col, u, cand);
        const uint32_t Wd = (d + 31) >> 5;
        if (P.hash_words)
            build_bitmap_hashed<BLOCK>(rp, col, cand, d, Wd, bm, tab, hash_bits_for(d));
        else
            build_bitmap<BLOCK>(rp, col, cand, d, Wd, bm);
        if (!compact) {
            // groups claim level-2 subtrees of this root, then share the deep ones
            if (threadIdx.x == 0) {
                ss.idle = 0;
                ss.active = BLOCK / G;
                ss.queued = 0;
                for (int x = 0; x < QCAP; ++x) ss.state[x] = 0;
            }
            __syncthreads();
            const uint32_t rem0 = k - 2;
            // small trees (k <= 4, vertex-centric): a group claims a few
            // tasks at a time; otherwise one task (one root edge) per claim
            const uint32_t claim = (k <= 4 && !EC) ? max(1u, d / (4u * (BLOCK / G))) : 1u;
            for (;;) {
                uint32_t t0 = 0;
                // without helpers (help_min = 0) the root's tasks are this
                // block's alone and are claimed in shared memory
                if (gl == 0) t0 = P.help_min ? atomicAdd(&P.task_next[s], claim) : atomicAdd(&sh.task, claim);
                t0 = __shfl_sync(gm, t0, leader);
                if (t0 >= d) break;
                const uint32_t t1 = min(t0 + claim, d);
                for (uint32_t t = t0; t < t1; ++t) walk_task<G>(P, bm, Wd, t, rem0, stk, acc, &ss, qwords, W0);
                int to = 0;
                if (gl == 0) to = timed_out(P.ctl);
                if (__shfl_sync(gm, to, leader)) break;
            }
            while (steal_or_finish<G>(P, &ss, qwords, W0, Wd, own, m))
                walk_frame<G>(P, bm, Wd, own, m[0], m[1], m[3], m[2], stk, acc, &ss, qwords, W0);
        } else {
            // one root edge u -> cand[i] at a time: compact C ∩ N+(cand[i]) and
            // let the groups claim its level-3 subtrees
            const uint32_t rem0 = k - 3;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (;;) {
                if (threadIdx.x == 0) {
                    uint32_t i = timed_out(P.ctl) ? NONE
                                                  : (P.help_min ? atomicAdd(&P.task_next[s], 1u) : atomicAdd(&sh.task, 1u));
                    sh.edge = (i != NONE && i < d) ? i : NONE;
                    sh.sub_next = 0;
                    ss.idle = 0;
                    ss.active = BLOCK / G;
                    ss.queued = 0;
                    for (int x = 0; x < QCAP; ++x) ss.state[x] = 0;
                }
                __syncthreads();
                const uint32_t i = sh.edge;
                if (i == NONE) break;
                const uint32_t* Ri = bm + (size_t)i * Wd;
                // word prefix popcounts of row i (the members of the edge's candidate set)
                if (warp == 0) {
                    uint32_t carry = 0;
                    for (uint32_t w0 = 0; w0 < Wd; w0 += 32) {
                        uint32_t w = w0 + lane;
                        uint32_t c = w < Wd ? __popc(Ri[w]) : 0;
                        uint32_t incl = c;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += y;
                        }
                        if (w < Wd) wpre[w] = carry + incl - c;
                        carry += __shfl_sync(0xffffffffu, incl, 31);
                    }
                    if (lane == 0) wpre[Wd] = carry;
                }
                __syncthreads();
                const uint32_t de = wpre[Wd];
                if (de + 2 < k) {
                    __syncthreads();
                    continue;
                }
                const uint32_t We = (de + 31) >> 5;
                // member list: positions of the set bits of row i
                for (uint32_t w = threadIdx.x; w < Wd; w += BLOCK) {
                    uint32_t bits = Ri[w], o = wpre[w];
                    while (bits) {
                        subidx[o++] = (w << 5) + (__ffs(bits) - 1);
                        bits &= bits - 1;
                    }
                }
                for (uint32_t x = threadIdx.x; x < de * We; x += BLOCK) sub[x] = 0;
                __syncthreads();
                // compacted rows: bit b of row a iff member b is an out-neighbour of member a
                for (uint32_t a = warp; a < de; a += NWARPS) {
                    const uint32_t pa = subidx[a];
                    const uint32_t* Ra = bm + (size_t)pa * Wd;
                    uint32_t* out = sub + (size_t)a * We;
                    for (uint32_t w = (pa >> 5) + lane; w < Wd; w += 32) {
                        uint32_t bits = Ra[w] & Ri[w];
                        while (bits) {
                            uint32_t bitpos = __ffs(bits) - 1;
                            bits &= bits - 1;
                            uint32_t b = wpre[w] + __popc(Ri[w] & ((1u << bitpos) - 1u));
                            atomicOr(&out[b >> 5], 1u << (b & 31));
                        }
                    }
                }
                __syncthreads();
                for (;;) {
                    uint32_t t = 0;
                    if (gl == 0) t = atomicAdd(&sh.sub_next, 1u);
                    t = __shfl_sync(gm, t, leader);
                    if (t >= de) break;
                    walk_task<G>(P, sub, We, t, rem0, stk, acc, &ss, qwords, W0);
                }
                while (steal_or_finish<G>(P, &ss, qwords, W0, We, own, m))
                    walk_frame<G>(P, sub, We, own, m[0], m[1], m[3], m[2], stk, acc, &ss, qwords, W0);
                __syncthreads();
            }
        }
    }
}

// Big roots of a single-graph launch: own a new root while any is left, then
// join roots with unclaimed tasks (P.help_min != 0).
template <int G, bool EC>
__device__ void block_phase(const CountParams& P, uint32_t* smem, BlockShared& sh, StealShared& ss, Acc& acc) {
    WorkCtl* wc = reinterpret_cast<WorkCtl*>(P.ctl + 1);
    int phase = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            sh.slot = next_big_slot(P, wc, phase);
            sh.task = 0;
        }
        __syncthreads();
        const uint32_t s = sh.slot;
        if (s == NONE) break;
        block_root<G, EC>(P, P.rp, P.col, P.k, s, P.roots[s], smem, sh, ss, acc);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------

template <int G, bool EC>
__global__ void __launch_bounds__(BLOCK) k_count_orient(const CountParams P) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ BlockShared sh;
    __shared__ StealShared ss;
    Acc acc;
    if (P.n_big > 0) block_phase<G, EC>(P, smem, sh, ss, acc);
    __syncthreads();
    if (P.n_work > P.n_big) {
        WarpShared* ws = reinterpret_cast<WarpShared*>(smem) + (threadIdx.x >> 5);
        warp_phase(P, *ws, acc);
    }
    // warp reduction (exact 128-bit), then one atomic pair per warp
    unsigned long long lo = acc.lo, hi = acc.hi, words = acc.words;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, lo, o);
        unsigned long long yh = __shfl_xor_sync(0xffffffffu, hi, o);
        words += __shfl_xor_sync(0xffffffffu, words, o);
        unsigned long long s = lo + y;
        hi += yh + (s < lo ? 1ull : 0ull);
        lo = s;
    }
    if ((threadIdx.x & 31) == 0) {
        add_u128(&P.ctl->total_lo, &P.ctl->total_hi, lo);
        if (hi) atomicAdd(&P.ctl->total_hi, hi);
        atomicAdd(&P.ctl->words, words);
        if (P.sm_work) {
            const unsigned sm = smid();
            if (sm < SM_WORK_SLOTS) atomicAdd(&P.sm_work[sm], words);
        }
    }
}

__global__ void k_finalize(const Ctl* ctl, kc_result* out) {
    kc_result r;
    r.total = ctl->total_lo;
    r.total_hi = ctl->total_hi;
    r.flags = ctl->flags | (ctl->total_hi ? KC_FLAG_TOTAL_OVERFLOW : 0u);
    r.status = (ctl->flags & KC_FLAG_TIMEOUT) ? KC_E_TIMEOUT : ((ctl->flags & KC_FLAG_INTERNAL) ? KC_E_INTERNAL : KC_OK);
    r.words = ctl->words;
    *out = r;
}

__global__ void k_write_result(kc_result* out, unsigned long long lo) {
    kc_result r;
    r.total = lo;
    r.total_hi = 0;
    r.flags = 0;
    r.status = KC_OK;
    r.words = 0;
    *out = r;
}

__global__ void k_set_deadline(Ctl* ctl, unsigned long long budget_ns) {
    ctl->deadline = budget_ns ? globaltimer_ns() + budget_ns : 0ull;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef void (*CountKernel)(const CountParams);

template <bool EC>
static CountKernel pick(uint32_t G) {
    switch (G) {
        case 1: return k_count_orient<1, EC>;
        case 2: return k_count_orient<2, EC>;
        case 4: return k_count_orient<4, EC>;
        case 8: return k_count_orient<8, EC>;
        case 16: return k_count_orient<16, EC>;
        default: return k_count_orient<32, EC>;
    }
}

static constexpr size_t SMEM_LIMIT = 220 * 1024;

struct Geometry {
    uint32_t dcap, wcap, depth;
    int in_smem;
    size_t smem_bytes;
    size_t gscratch_words;
    uint32_t hash_words;
};

// 16-bit slots of the candidate position table for candidate sets up to dcap
static uint32_t hash_words_for(uint32_t dcap) { return hash_table_words(dcap); }

static Geometry plan_geometry(uint32_t dcap, uint32_t k, uint32_t G, bool ec) {
    Geometry g;
    g.dcap = std::max<uint32_t>(dcap, 1);
    g.wcap = (g.dcap + 31) / 32;
    // stack levels: the DFS pushes while rem >= 3, i.e. rem0 - 2 levels
    const bool ec_compact = ec && k >= EC_COMPACT_MIN_K;
    const uint32_t rem0 = ec_compact ? k - 3 : (k > 2 ? k - 2 : 0);
    g.depth = rem0 > 2 ? rem0 - 2 : 1;
    const size_t D0 = (g.dcap + 31) & ~31u;
    size_t region = (size_t)g.dcap * g.wcap;                        // bitmap
    if (ec_compact) region += (size_t)g.dcap * g.wcap + D0 + g.wcap + 32;  // sub-bitmap, members, prefixes
    region += (size_t)QCAP * g.wcap;                                // donated frames
    region += (size_t)(BLOCK / G) * (g.depth + 1) * g.wcap;        // per group: taken frame + child lists
    const size_t warp_bytes = sizeof(WarpShared) * NWARPS;
    const size_t hw = g.dcap < 65535 ? hash_words_for(g.dcap) : 0;
    g.hash_words = 0;
    if (hw && (D0 + region + hw) * 4 <= SMEM_LIMIT) {
        g.in_smem = 1;
        g.hash_words = (uint32_t)hw;
        g.smem_bytes = (D0 + region + hw) * 4;
        g.gscratch_words = 0;
    } else if ((D0 + region) * 4 <= SMEM_LIMIT) {
        g.in_smem = 1;
        g.smem_bytes = (D0 + region) * 4;
        g.gscratch_words = 0;
    } else {
        g.in_smem = 0;
        g.smem_bytes = D0 * 4;
        g.gscratch_words = (region + 63) & ~(size_t)63;
    }
    g.smem_bytes = std::max(g.smem_bytes, warp_bytes);
    return g;
}

int sm_count_of_current_device() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static uint64_t roots_with_outdeg_at_least(const kc_graph* g, uint64_t dmin) {
    uint64_t c = 0;
    for (uint64_t d = dmin; d < g->outdeg_hist.size(); ++d) c += g->outdeg_hist[d];
    return c;
}

size_t ctl_bytes() { return sizeof(Ctl) + sizeof(WorkCtl) + 256; }

static kc_status plan_launch(kc_graph* g, uint32_t k, uint32_t G, bool ec, Geometry& geo, int& blocks,
                             CountKernel& kern) {
    geo = plan_geometry(g->d_max, k, G, ec);
    kern = ec ? pick<true>(G) : pick<false>(G);
    KC_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem_bytes));
    int bps = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BLOCK, geo.smem_bytes));
    if (bps < 1) return set_error(KC_E_UNSUPPORTED, "count kernel cannot be resident (smem %zu)", geo.smem_bytes);
    blocks = bps * g->sm_count;
    return KC_OK;
}

kc_status count_reserve(kc_graph* g, uint32_t k_max, int pivot, int per_vertex, cudaStream_t s) {
    (void)pivot;
    (void)s;
    if (per_vertex) KC_CHECK(dev_alloc(g->pv, ((size_t)g->n + 16) * 8));
    KC_CHECK(dev_alloc(g->ctl, ctl_bytes()));
    KC_CHECK(dev_alloc(g->sm_work, SM_WORK_SLOTS * 8));
    size_t need = 64;
    for (uint32_t k = 3; k <= std::min<uint32_t>(k_max, LIST_MAX_K); ++k) need = std::max(need, list_scratch_words(g, k) + 64);
    for (uint32_t G : {1u, 2u, 4u, 8u, 16u, 32u})
        for (int ec = 0; ec < 2; ++ec)
            for (uint32_t k = 3; k <= std::min<uint32_t>(k_max, MAX_DEPTH + 4); ++k) {
                Geometry geo;
                int blocks = 0;
                CountKernel kern;
                KC_CHECK(plan_launch(g, k, G, ec != 0, geo, blocks, kern));
                need = std::max(need, geo.gscratch_words * blocks + 64);
                for (int pv = 0; pv < 2; ++pv)
                    if (deep_supported(g, k, pv != 0) && (pv == 0 || per_vertex)) {
                        size_t sw = 0;
                        KC_CHECK(deep_plan(g, k, ec != 0, pv != 0, &sw, &blocks));
                        need = std::max(need, sw + 64);
                    }
            }
    KC_CHECK(dev_alloc(g->scratch, need * 4));
    KC_CHECK(dev_alloc(g->tmp, (2 * (size_t)g->n + 64) * 4));
    return KC_OK;
}

kc_status count_launch(kc_graph* g, const CountArgs& a, kc_result* result_dev, cudaStream_t s) {
    const uint32_t k = a.k;
    KC_CHECK(dev_alloc(g->ctl, ctl_bytes()));
    Ctl* ctl = (Ctl*)g->ctl.ptr;
    KC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl) + sizeof(WorkCtl), s));
    KC_CHECK(dev_alloc(g->sm_work, SM_WORK_SLOTS * 8));
    unsigned long long* sm_work = (unsigned long long*)g->sm_work.ptr;
    KC_CUDA(cudaMemsetAsync(sm_work, 0, SM_WORK_SLOTS * 8, s));
    if (k <= 2 || (uint64_t)k > (uint64_t)g->d_max + 1) {
        unsigned long long v = k == 1 ? g->n : (k == 2 ? g->m : 0ull);
        k_write_result<<<1, 1, 0, s>>>(result_dev, v);
        note_launch();
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    if (k > MAX_DEPTH + 4)
        return set_error(KC_E_UNSUPPORTED, "orientation traversal supports k <= %d; use pivoting for larger k",
                         MAX_DEPTH + 4);
    unsigned long long budget = g->time_limit_s > 0 ? (unsigned long long)(g->time_limit_s * 1e9) : 0ull;
    if (a.scheme == KC_SCHEME_VC_LIST || a.scheme == KC_SCHEME_EC_LIST) {
        // the traversal on sorted lists (no binary encoding)
        if (a.per_vertex_dev) return set_error(KC_E_UNSUPPORTED, "the list traversal gives totals only");
        k_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
        note_launch();
        KC_CUDA(cudaGetLastError());
        WorkCtl* wc = reinterpret_cast<WorkCtl*>(ctl + 1);
        KC_CHECK(list_launch(g, k, a.scheme == KC_SCHEME_EC_LIST, ctl, &wc->root_cursor, sm_work, s));
        k_finalize<<<1, 1, 0, s>>>(ctl, result_dev);
        note_launch();
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    const bool ec = a.scheme == KC_SCHEME_EC;
    const uint32_t G = a.subwarp;
    const uint64_t n_work = roots_with_outdeg_at_least(g, k - 1);
    const uint64_t n_big = roots_with_outdeg_at_least(g, std::max<uint64_t>(SMALL_D + 1, k - 1));
    const bool pv = a.per_vertex_dev != nullptr;
    if (pv && !deep_supported(g, k, true))
        return set_error(KC_E_UNSUPPORTED, "per-vertex counts in orientation mode need 3 <= k <= 36");
    if (deep_supported(g, k, pv)) {
        // k >= 5, or per-vertex counts: the traversal with re-encoded small nodes (kc_deep.cu)
        size_t sw = 0;
        int dblocks = 0;
        KC_CHECK(deep_plan(g, k, ec && !(pv && k < 4), pv, &sw, &dblocks));
        KC_CHECK(dev_alloc(g->scratch, (sw + 64) * 4));
        KC_CHECK(dev_alloc(g->tmp, (2 * (size_t)g->n + 64) * 4));
        unsigned long long* pvacc = nullptr;
        if (pv) {
            KC_CHECK(dev_alloc(g->pv, ((size_t)g->n + 16) * 8));
            pvacc = (unsigned long long*)g->pv.ptr;
            KC_CUDA(cudaMemsetAsync(pvacc, 0, (size_t)g->n * 8, s));
        }
        uint32_t* task_next = (uint32_t*)g->tmp.ptr;
        uint32_t* task_total = task_next + n_big;
        if (n_big) KC_CUDA(cudaMemsetAsync(task_next, 0, (size_t)n_big * 8, s));
        k_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
        note_launch();
        KC_CUDA(cudaGetLastError());
        if (n_work > 0)
            KC_CHECK(deep_launch(g, k, ec, (uint32_t)n_big, (uint32_t)n_work, task_next, task_total,
                                 (uint32_t*)g->scratch.ptr, pvacc, ctl, s));
        if (pv) KC_CHECK(pv_to_input(g, pvacc, a.per_vertex_dev, s));
        k_finalize<<<1, 1, 0, s>>>(ctl, result_dev);
        note_launch();
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    Geometry geo;
    int blocks = 0;
    CountKernel kern;
    KC_CHECK(plan_launch(g, k, G, ec, geo, blocks, kern));
    KC_CHECK(dev_alloc(g->scratch, (geo.gscratch_words * blocks + 64) * 4));
    KC_CHECK(dev_alloc(g->tmp, ((size_t)g->n + 64) * 4));
    CountParams P;
    memset(&P, 0, sizeof(P));
    P.rp = (const uint32_t*)g->row_ptr.ptr;
    P.col = (const uint32_t*)g->col.ptr;
    P.k = k;
    P.roots = (const uint32_t*)g->roots.ptr;
    P.n_big = (uint32_t)n_big;
    P.n_work = (uint32_t)n_work;
    P.task_next = (uint32_t*)g->tmp.ptr;
    // small trees (k <= 4): a root stays with its block and groups claim a
    // few tasks at a time; deeper trees: one task per claim, and idle blocks
    // join roots that still have unclaimed tasks
    P.help_min = k <= 4 ? 0u : 2u;
    P.dcap = geo.dcap;
    P.wcap = geo.wcap;
    P.depth = geo.depth;
    P.in_smem = geo.in_smem;
    P.gscratch = (uint32_t*)g->scratch.ptr;
    P.gscratch_words = geo.gscratch_words;
    P.hash_words = geo.hash_words;
    P.ctl = ctl;
    P.sm_work = sm_work;
    if (n_big) KC_CUDA(cudaMemsetAsync(g->tmp.ptr, 0, (size_t)n_big * 4, s));
    k_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
    note_launch();
    KC_CUDA(cudaGetLastError());
    if (n_work > 0) {
        kern<<<blocks, BLOCK, geo.smem_bytes, s>>>(P);
        note_launch();
        KC_CUDA(cudaGetLastError());
    }
    k_finalize<<<1, 1, 0, s>>>(ctl, result_dev);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}


kc_status list_cliques_launch(kc_graph* g, uint32_t k, uint32_t* out, uint64_t cap, kc_result* result_dev,
                              cudaStream_t s) {
    if (k < 3 || k > LIST_MAX_K) return set_error(KC_E_UNSUPPORTED, "listing takes 3 <= k <= %u", LIST_MAX_K);
    KC_CHECK(dev_alloc(g->ctl, ctl_bytes()));
    Ctl* ctl = (Ctl*)g->ctl.ptr;
    WorkCtl* wc = reinterpret_cast<WorkCtl*>(ctl + 1);
    // the cliques-found counter sits right after the work counters
    unsigned long long* emitted = reinterpret_cast<unsigned long long*>(wc + 1);
    KC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl) + sizeof(WorkCtl) + sizeof(unsigned long long), s));
    KC_CHECK(dev_alloc(g->sm_work, SM_WORK_SLOTS * 8));
    unsigned long long* sm_work = (unsigned long long*)g->sm_work.ptr;
    KC_CUDA(cudaMemsetAsync(sm_work, 0, SM_WORK_SLOTS * 8, s));
    const unsigned long long budget = g->time_limit_s > 0 ? (unsigned long long)(g->time_limit_s * 1e9) : 0ull;
    k_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
    note_launch();
    KC_CUDA(cudaGetLastError());
    if ((uint64_t)k <= (uint64_t)g->d_max + 1)
        KC_CHECK(list_launch(g, k, false, ctl, &wc->root_cursor, sm_work, s, out, cap, emitted));
    k_finalize<<<1, 1, 0, s>>>(ctl, result_dev);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// ---------------------------------------------------------------------------
// Batched counts: many (graph, k) queries in one persistent launch.  The
// item space is every query's roots with out-degree >= k - 1: first the big
// roots of all queries (one block each, as block_root), then the small ones
// (one warp each, as warp_root).  Each query accumulates an exact 128-bit
// total of its own.
// ---------------------------------------------------------------------------
struct BatchCtl {
    unsigned big_cursor;
    unsigned small_cursor;
};

struct BatchParams {
    CountParams base;           // geometry and control record (graph fields unused)
    const QDesc* q;
    uint32_t nq;
    uint32_t chunk;             // small roots per claim
    const uint32_t* nbig;       // per query: roots with more than 32 candidates
    const uint32_t* big_pre;    // exclusive prefix sums, nq + 1 entries
    const uint32_t* small_pre;
    unsigned long long* out;    // per query: total low, total high, words
    BatchCtl* bc;
    unsigned* remaining;        // per query: roots not yet completed
    kc_result* early;           // nullable: each query's result as soon as it completes (by slot)
    unsigned* done;             // with early: set to 1 (after a system fence) once early[slot] is written
};

// a query's result from its accumulators; `complete`: every root finished
__device__ __forceinline__ kc_result compose_result(const QDesc& D, const unsigned long long* out3, bool complete) {
    kc_result r;
    r.total = 0;
    r.total_hi = 0;
    r.flags = 0;
    r.status = KC_OK;
    r.words = 0;
    if (D.k == 1) {
        r.total = D.n;
    } else if (D.k == 2) {
        r.total = D.m;
    } else if (D.k <= D.d_max + 1) {
        r.total = *(volatile const unsigned long long*)&out3[0];
        r.total_hi = *(volatile const unsigned long long*)&out3[1];
        r.words = *(volatile const unsigned long long*)&out3[2];
        if (r.total_hi) r.flags |= KC_FLAG_TOTAL_OVERFLOW;
    }
    if (!complete) {
        r.flags |= KC_FLAG_TIMEOUT;
        r.status = KC_E_TIMEOUT;
    }
    return r;
}

// publish query q's result early (one thread; every contribution is in out)
__device__ __forceinline__ void publish_early(const BatchParams& B, uint32_t q) {
    const QDesc& D = B.q[q];
    __threadfence();
    B.early[D.slot] = compose_result(D, B.out + 3 * (size_t)q, true);
    __threadfence_system();
    *(volatile unsigned*)&B.done[D.slot] = 1u;
}

// `n` more roots of query q are complete (one thread, after their counts
// were added to out)
__device__ __forceinline__ void complete_roots(const BatchParams& B, uint32_t q, uint32_t n) {
    if (n == 0) return;
    __threadfence();
    if (atomicSub(&B.remaining[q], n) == n && B.early) publish_early(B, q);
}

// the query whose item range [pre[q], pre[q + 1]) holds item i (i < pre[nq])
__device__ __forceinline__ uint32_t find_query(const uint32_t* pre, uint32_t nq, uint32_t i) {
    uint32_t lo = 0, hi = nq;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid + 1] <= i) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// exact warp sum of the lanes' partials into out3 (all 32 lanes call it)
__device__ __forceinline__ void flush_warp_acc(Acc& acc, unsigned long long* out3) {
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
    if ((threadIdx.x & 31) == 0) {
        add_u128(&out3[0], &out3[1], lo);
        if (hi) atomicAdd(&out3[1], hi);
        if (words) atomicAdd(&out3[2], words);
    }
    acc = Acc();
}

// roots (decreasing out-degree) with out-degree >= t
__device__ __forceinline__ uint32_t roots_at_least(const uint32_t* rp, const uint32_t* roots, uint32_t n, uint32_t t) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t r = roots[mid];
        if (rp[r + 1] - rp[r] >= t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_batch_prep(const BatchParams B, uint32_t* __restrict__ nwork) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.nq) return;
    const QDesc D = B.q[i];
    uint32_t* nbig = const_cast<uint32_t*>(B.nbig);
    if (D.k < 3 || D.k > D.d_max + 1) {
        nbig[i] = nwork[i] = 0;
        B.remaining[i] = 0;
        if (B.early) publish_early(B, i);  // nothing to traverse
        return;
    }
    const uint32_t w = roots_at_least(D.rp, D.roots, D.n_roots, D.k - 1);
    nwork[i] = w;
    nbig[i] = roots_at_least(D.rp, D.roots, D.n_roots, max(D.k - 1, (uint32_t)SMALL_D + 1));
    B.remaining[i] = w;
    if (w == 0 && B.early) publish_early(B, i);
}

// exclusive prefix sums of nbig and of nwork - nbig (one block of 1024)
__global__ void __launch_bounds__(1024) k_batch_scan(const uint32_t* __restrict__ nbig,
                                                      const uint32_t* __restrict__ nwork, uint32_t nq,
                                                      uint32_t* __restrict__ big_pre, uint32_t* __restrict__ small_pre) {
    __shared__ uint32_t wb[32], wsm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t cb = 0, cs = 0;
    for (uint32_t base = 0; base < nq; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t b = i < nq ? nbig[i] : 0, sm = i < nq ? nwork[i] - nbig[i] : 0;
        uint32_t ib = b, is = sm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yb = __shfl_up_sync(0xffffffffu, ib, o), ys = __shfl_up_sync(0xffffffffu, is, o);
            if (lane >= o) {
                ib += yb;
                is += ys;
            }
        }
        if (lane == 31) {
            wb[warp] = ib;
            wsm[warp] = is;
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t xb = wb[lane], xs = wsm[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t yb = __shfl_up_sync(0xffffffffu, xb, o), ys = __shfl_up_sync(0xffffffffu, xs, o);
                if (lane >= o) {
                    xb += yb;
                    xs += ys;
                }
            }
            wb[lane] = xb;
            wsm[lane] = xs;
        }
        __syncthreads();
        const uint32_t ob = cb + (warp ? wb[warp - 1] : 0u) + ib - b;
        const uint32_t os = cs + (warp ? wsm[warp - 1] : 0u) + is - sm;
        if (i < nq) {
            big_pre[i] = ob;
            small_pre[i] = os;
        }
        cb += wb[31];
        cs += wsm[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        big_pre[nq] = cb;
        small_pre[nq] = cs;
    }
}

// Big roots of a batched launch, one per block, until none is left.
template <int G, bool EC>
__device__ void batch_big(const BatchParams& B, uint32_t* smem, BlockShared& sh, StealShared& ss, uint32_t* s_qu,
                          Acc& acc) {
    const uint32_t nbig_total = B.big_pre[B.nq];
    while (nbig_total) {
        if (threadIdx.x == 0) {
            const uint32_t i = timed_out(B.base.ctl) ? NONE : atomicAdd(&B.bc->big_cursor, 1u);
            uint32_t q = NONE, u = 0;
            if (i < nbig_total) {
                q = find_query(B.big_pre, B.nq, i);
                u = B.q[q].roots[i - B.big_pre[q]];
            }
            s_qu[0] = q;
            s_qu[1] = u;
            sh.task = 0;
        }
        __syncthreads();
        const uint32_t q = s_qu[0];
        if (q == NONE) break;
        const QDesc* D = B.q + q;
        block_root<G, EC>(B.base, D->rp, D->col, D->k, 0, s_qu[1], smem, sh, ss, acc);
        flush_warp_acc(acc, B.out + 3 * (size_t)q);
        __syncthreads();
        if (threadIdx.x == 0 && !timed_out(B.base.ctl)) complete_roots(B, q, 1);
    }
    __syncthreads();
}

// Small roots of a batched launch, one per warp, `chunk` per claim.
__device__ void batch_small(const BatchParams& B, uint32_t* smem, Acc& acc) {
    const uint32_t nsmall_total = B.small_pre[B.nq];
    if (nsmall_total == 0) return;
    WarpShared* ws = reinterpret_cast<WarpShared*>(smem) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    uint32_t cur = NONE, lo = 0, hi = 0;  // the current query and its item range
    uint32_t finished = 0;                 // roots of cur completed since its last flush
    for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = timed_out(B.base.ctl) ? NONE : atomicAdd(&B.bc->small_cursor, B.chunk);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= nsmall_total) break;
        const uint32_t j1 = min(j + B.chunk, nsmall_total);
        bool stop = false;
        for (uint32_t t = j; t < j1; ++t) {
            if (t < lo || t >= hi) {
                const uint32_t q = find_query(B.small_pre, B.nq, t);
                if (cur != NONE) {
                    flush_warp_acc(acc, B.out + 3 * (size_t)cur);
                    if (lane == 0) complete_roots(B, cur, finished);
                }
                finished = 0;
                cur = q;
                lo = B.small_pre[q];
                hi = B.small_pre[q + 1];
            }
            const QDesc* D = B.q + cur;
            warp_root(B.base, D->rp, D->col, D->k, D->roots[B.nbig[cur] + (t - lo)], *ws, acc);
            int to = 0;
            if (lane == 0) to = timed_out(B.base.ctl);
            if (__shfl_sync(0xffffffffu, to, 0)) {
                stop = true;
                break;
            }
            ++finished;
        }
        if (stop) break;
        // a query whose last roots this warp holds is published without waiting
        // for the warp's next claim
        if (cur != NONE && finished && hi <= j1) {
            flush_warp_acc(acc, B.out + 3 * (size_t)cur);
            if (lane == 0) complete_roots(B, cur, finished);
            finished = 0;
        }
    }
    if (cur != NONE) {
        flush_warp_acc(acc, B.out + 3 * (size_t)cur);
        if (lane == 0 && !timed_out(B.base.ctl)) complete_roots(B, cur, finished);
    }
}

// Odd blocks take the small roots first and even blocks the big ones, so
// that neither kind waits for the other; queries are ordered cheapest first
// by the host, so light queries complete early in both phases.
template <int G, bool EC>
__global__ void __launch_bounds__(BLOCK) k_count_batch(const BatchParams B) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ BlockShared sh;
    __shared__ StealShared ss;
    __shared__ uint32_t s_qu[2];
    Acc acc;
    if (blockIdx.x & 1) {
        batch_small(B, smem, acc);
        __syncthreads();
        batch_big<G, EC>(B, smem, sh, ss, s_qu, acc);
    } else {
        batch_big<G, EC>(B, smem, sh, ss, s_qu, acc);
        batch_small(B, smem, acc);
    }
}

__global__ void k_batch_finalize(const QDesc* __restrict__ q, uint32_t nq, const unsigned long long* __restrict__ out,
                                 const unsigned* __restrict__ remaining, kc_result* __restrict__ res) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const QDesc D = q[i];
    res[D.slot] = compose_result(D, out + 3 * (size_t)i, remaining[i] == 0);
}

typedef void (*BatchKernel)(const BatchParams);

template <bool EC>
static BatchKernel pick_batch(uint32_t G) {
    switch (G) {
        case 1: return k_count_batch<1, EC>;
        case 2: return k_count_batch<2, EC>;
        case 4: return k_count_batch<4, EC>;
        case 8: return k_count_batch<8, EC>;
        case 16: return k_count_batch<16, EC>;
        default: return k_count_batch<32, EC>;
    }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t batch_ws_bytes(uint32_t nq) {
    return al256(sizeof(Ctl) + sizeof(BatchCtl)) + 5 * al256(((size_t)nq + 1) * 4) + al256((size_t)nq * 24 + 8);
}

size_t batch_smem_bytes(uint32_t d_cap, uint32_t k_max, const BatchConfig& cfg) {
    const Geometry geo = plan_geometry(std::max<uint32_t>(d_cap, 1), std::max<uint32_t>(k_max, 3), cfg.subwarp,
                                       cfg.ec != 0);
    return geo.in_smem ? geo.smem_bytes : 0;
}

kc_status batch_launch(const QDesc* q_dev, uint32_t nq, uint32_t d_cap, uint32_t k_max, const BatchConfig& cfg,
                       void* ws, double time_limit_s, int sm_count, kc_result* results_dev, kc_result* early,
                       unsigned* done, cudaStream_t s) {
    if (nq == 0) return KC_OK;
    const uint32_t G = cfg.subwarp;
    if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32)
        return set_error(KC_E_INVALID_ARG, "subwarp must be 1, 2, 4, 8, 16 or 32");
    if (k_max > MAX_DEPTH + 4)
        return set_error(KC_E_UNSUPPORTED, "orientation traversal supports k <= %d", MAX_DEPTH + 4);
    if ((early == nullptr) != (done == nullptr)) return set_error(KC_E_INVALID_ARG, "early and done go together");
    char* p = (char*)ws;
    Ctl* ctl = (Ctl*)p;
    BatchCtl* bc = (BatchCtl*)(ctl + 1);
    p += al256(sizeof(Ctl) + sizeof(BatchCtl));
    uint32_t* arr[5];
    for (int i = 0; i < 5; ++i) {
        arr[i] = (uint32_t*)p;
        p += al256(((size_t)nq + 1) * 4);
    }
    uint32_t *nbig = arr[0], *nwork = arr[1], *big_pre = arr[2], *small_pre = arr[3], *remaining = arr[4];
    unsigned long long* out = (unsigned long long*)p;
    KC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl) + sizeof(BatchCtl), s));
    KC_CUDA(cudaMemsetAsync(out, 0, (size_t)nq * 24, s));
    BatchParams B;
    memset(&B, 0, sizeof(B));
    B.base.ctl = ctl;
    B.base.help_min = 0;
    B.base.in_smem = 1;
    B.q = q_dev;
    B.nq = nq;
    B.chunk = std::max<uint32_t>(cfg.chunk, 1);
    B.nbig = nbig;
    B.big_pre = big_pre;
    B.small_pre = small_pre;
    B.out = out;
    B.bc = bc;
    B.remaining = remaining;
    B.early = early;
    B.done = done;
    const unsigned qb = (nq + 255) / 256;
    k_batch_prep<<<qb, 256, 0, s>>>(B, nwork);
    note_launch();
    k_batch_scan<<<1, 1024, 0, s>>>(nbig, nwork, nq, big_pre, small_pre);
    note_launch();
    const unsigned long long budget = time_limit_s > 0 ? (unsigned long long)(time_limit_s * 1e9) : 0ull;
    k_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
    note_launch();
    KC_CUDA(cudaGetLastError());
    if (k_max >= 3 && d_cap >= 2) {
        const Geometry geo = plan_geometry(d_cap, k_max, G, cfg.ec != 0);
        if (!geo.in_smem)
            return set_error(KC_E_UNSUPPORTED, "batched launches need out-degrees whose bitmaps fit in shared "
                                               "memory (largest out-degree %u)", d_cap);
        BatchKernel kern = cfg.ec ? pick_batch<true>(G) : pick_batch<false>(G);
        KC_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)geo.smem_bytes));
        int bps = 0;
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BLOCK, geo.smem_bytes));
        if (bps < 1) return set_error(KC_E_UNSUPPORTED, "batch kernel cannot be resident (smem %zu)", geo.smem_bytes);
        B.base.dcap = geo.dcap;
        B.base.wcap = geo.wcap;
        B.base.depth = geo.depth;
        B.base.hash_words = geo.hash_words;
        kern<<<bps * sm_count, BLOCK, geo.smem_bytes, s>>>(B);
        note_launch();
        KC_CUDA(cudaGetLastError());
    }
    k_batch_finalize<<<qb, 256, 0, s>>>(q_dev, nq, out, remaining, results_dev);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

}  // namespace kc

// ---------------------------------------------------------------------------
// Counting without device allocation.
//
// kc_count_async takes its working memory (control words, per-root task
// counters, and global-memory bitmaps for very large candidate sets) from
// the graph handle, allocating it on first use.  Some callers cannot let a
// library allocate: their device memory is entirely owned by another
// allocator (a framework's caching pool, a pre-partitioned arena), or they
// cannot afford the device-wide synchronisation that cudaFree implies in a
// latency-critical loop.  kc_count_noalloc runs the same kernel with its
// scratch in the fixed array below instead.
// ---------------------------------------------------------------------------
namespace kc {

static constexpr size_t NOALLOC_WORDS = (size_t)1 << 20;  // 4 MiB, resident on every device that loads the library
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];
static constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of the array, per device (set up once)
static std::mutex g_noalloc_mu;                      // host threads that set up a device together

}  // namespace kc

extern "C" kc_status kc_count_noalloc(const kc_graph* g, uint32_t k, int scheme, uint32_t subwarp,
                                      kc_result* result_dev, void* stream) {
    using namespace kc;
    clear_error();
    if (!g) return set_error(KC_E_INVALID_ARG, "NULL graph");
    if (!result_dev) return set_error(KC_E_INVALID_ARG, "result_dev is NULL");
    if (k == 0) return set_error(KC_E_INVALID_ARG, "k must be >= 1");
    if (scheme != KC_SCHEME_AUTO && scheme != KC_SCHEME_VC && scheme != KC_SCHEME_EC)
        return set_error(KC_E_INVALID_ARG, "unknown scheme %d", scheme);
    if (subwarp != 0 && subwarp != 1 && subwarp != 2 && subwarp != 4 && subwarp != 8 && subwarp != 16 && subwarp != 32)
        return set_error(KC_E_INVALID_ARG, "subwarp must be 0, 1, 2, 4, 8, 16 or 32");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_error(KC_E_UNSUPPORTED, "device index %d too large", dev);
    if (dev != g->device) return set_error(KC_E_INVALID_ARG, "the graph lives on device %d, not %d", g->device, dev);
    uint32_t* scratch = nullptr;
    {
        // set-up, once per device, with that device current: the host-side name
        // of the array is not a device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* ptr = nullptr;
            KC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            g_noalloc_addr[dev] = ptr;
        }
        scratch = (uint32_t*)g_noalloc_addr[dev];
    }
    if (k <= 2 || (uint64_t)k > (uint64_t)g->d_max + 1) {
        unsigned long long v = k == 1 ? g->n : (k == 2 ? g->m : 0ull);
        k_write_result<<<1, 1, 0, s>>>(result_dev, v);
        note_launch();
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    if (k > MAX_DEPTH + 4)
        return set_error(KC_E_UNSUPPORTED, "orientation traversal supports k <= %d", MAX_DEPTH + 4);
    const bool ec = (scheme == KC_SCHEME_AUTO ? (k < 6 ? KC_SCHEME_VC : KC_SCHEME_EC) : scheme) == KC_SCHEME_EC;
    uint32_t G = subwarp ? subwarp : (((g->d_max + 31) / 32) <= 8 ? 4u : 8u);
    Geometry geo;
    int blocks = 0;
    CountKernel kern;
    KC_CHECK(plan_launch(const_cast<kc_graph*>(g), k, G, ec, geo, blocks, kern));
    if (!geo.in_smem)
        return set_error(KC_E_UNSUPPORTED,
                         "candidate sets of %u vertices need global-memory bitmaps; use kc_count_async", g->d_max);
    const uint64_t n_work = roots_with_outdeg_at_least(g, k - 1);
    const uint64_t n_big = roots_with_outdeg_at_least(g, std::max<uint64_t>(SMALL_D + 1, k - 1));
    const size_t ctl_words = ((sizeof(Ctl) + sizeof(WorkCtl) + 255) & ~(size_t)255) / 4;  // 256-byte aligned
    if (ctl_words + n_big > NOALLOC_WORDS)
        return set_error(KC_E_UNSUPPORTED, "%llu roots with more than 32 candidates exceed the %zu-word scratch array",
                         (unsigned long long)n_big, NOALLOC_WORDS - ctl_words);
    Ctl* ctl = (Ctl*)scratch;
    uint32_t* task_next = scratch + ctl_words;
    // the array keeps the previous call's contents: clear what must start at zero
    KC_CUDA(cudaMemsetAsync(scratch, 0, (ctl_words + n_big) * 4, s));
    CountParams P;
    memset(&P, 0, sizeof(P));
    P.rp = (const uint32_t*)g->row_ptr.ptr;
    P.col = (const uint32_t*)g->col.ptr;
    P.k = k;
    P.roots = (const uint32_t*)g->roots.ptr;
    P.n_big = (uint32_t)n_big;
    P.n_work = (uint32_t)n_work;
    P.task_next = task_next;
    P.help_min = k <= 4 ? 0u : 2u;
    P.dcap = geo.dcap;
    P.wcap = geo.wcap;
    P.depth = geo.depth;
    P.in_smem = 1;
    P.gscratch = nullptr;
    P.gscratch_words = 0;
    P.hash_words = geo.hash_words;
    P.ctl = ctl;
    unsigned long long budget = g->time_limit_s > 0 ? (unsigned long long)(g->time_limit_s * 1e9) : 0ull;
    k_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
    note_launch();
    KC_CUDA(cudaGetLastError());
    if (n_work > 0) {
        kern<<<blocks, BLOCK, geo.smem_bytes, s>>>(P);
        note_launch();
        KC_CUDA(cudaGetLastError());
    }
    k_finalize<<<1, 1, 0, s>>>(ctl, result_dev);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}
