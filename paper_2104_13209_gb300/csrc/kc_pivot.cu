// Pivoting k-clique counting (Fig. 3; Sections 2.3, 2.4, 3.2, 3.4, 3.5).
//
// Level 1 is oriented: root r has candidate set C = N+(r) (ascending library
// id).  Below it the search runs on the undirected sub-graph induced by C,
// binary encoded (Section 3.4): adj row i = {j : C[j] adjacent to C[i]}.
// A tree node holds the candidate set S (a bitmap; every member is adjacent
// to every vertex on the path), h held vertices (the root included) and q
// pivots on the path:
//   S empty            -> leaf (h, q): it stands for the C(q, j - h) cliques of
//                         size j made of the held vertices plus j - h pivots;
//   S a clique of size c -> leaf (h, q + c) (every further level would pick a
//                         pivot adjacent to all the rest);
//   otherwise          -> pivot p = the member of S with the most neighbours in S
//                         (ties: lowest index); for each x in S \ N(p), ascending:
//                         child S' = S ∩ N(x) minus the members of S \ N(p) before x,
//                         with x held (x != p) or a pivot (x == p).
// Fixed-k mode (Fig. 3's stopping criterion) skips children with more than k
// held vertices and subtrees that cannot reach size k.
//
// Leaves are counted in an (h, q) histogram (shared memory per block for small
// h and q, global memory otherwise); a final kernel turns it into per-size
// counts with an exact binomial table (64-bit values, saturation = overflow).  Per-vertex counts for one size k use subtree sums:
// a held vertex gains C(q, k - h) per leaf below it, a pivot C(q - 1, k - h - 1).
//
// Work distribution: big roots (|C| > 32) go to blocks in decreasing
// out-degree order; the block builds the bitmap, picks the root's pivot, and
// its warps claim the root's branch subtrees from a per-root counter in
// global memory (so other blocks can join a large root).  Each warp walks its
// subtree with warp-parallel pivot selection (lanes over the candidates); a
// node with at most 32 candidates is re-extracted into a sub-graph of one-word
// rows (Section 2.4: extraction can happen at any level).  Small roots run in
// warp mode, one warp per root.  Busy warps donate halves of their frames to
// idle warps of the block, or to idle blocks through a global queue.
#include <algorithm>

#include "kc_bitmap.cuh"
#include "kc_common.cuh"

namespace kc {

static constexpr int PB = 256;
static constexpr int PW = PB / 32;
static constexpr int PSMALL = 32;
static constexpr uint32_t HDR = 10;  // per-level header words: h, q, p, vtx, held, pad, sumH(2), sumP(2)
static constexpr unsigned long long SAT = ~0ull;

struct PivotParams {
    const uint32_t* rp;
    const uint32_t* col;
    const uint32_t* roots;       // library ids, decreasing out-degree
    uint32_t n_big;              // roots[0, n_big): |C| > 32
    uint32_t n_work;             // roots[n_big, n_work): 32 >= |C| >= dmin
    uint32_t n;                  // vertices (per-vertex accumulators)
    uint32_t* task_next;         // per big root: next unclaimed branch (zeroed)
    uint32_t kfix;               // 0 = every size; else only size kfix is needed
    uint32_t pvk;                // per-vertex size (0 = none)
    unsigned long long* pv;      // per-vertex accumulators (library numbering)
    const unsigned long long* binom;  // C(a, b), a, b < bstride, SAT = >= 2^64 - 1
    uint32_t bstride;
    unsigned long long* leaves;  // histogram [h * hq + q]
    uint32_t hq;
    uint32_t dcap, wcap;
    uint32_t lvl_cap;            // wide stack levels per warp
    uint32_t lvl_smem;           // of which kept in shared memory
    int adj_in_smem;
    uint32_t* gstack;            // per-warp wide stack levels beyond lvl_smem (global)
    size_t gstack_words;         // words per warp
    uint32_t* gadj;              // per-block adjacency when it does not fit in shared memory
    size_t gadj_words;
    uint32_t* gq;                // global frame queue: gq_cap slots of gq_stride words
    unsigned* gq_state;          // per slot: 0 empty, 1 being written, 2 ready, 3 being read
    uint32_t gq_cap, gq_stride;
    Ctl* ctl;
};

struct PWorkCtl {
    unsigned int root_cursor;
    unsigned int help_lo;
    unsigned int small_cursor;
    unsigned int g_idle;     // blocks waiting in the global frame pool
    unsigned int g_active;   // blocks not yet finished (set by the host to the grid size)
    unsigned int g_queued;   // frames ready in the global queue
    unsigned int pad[2];
};

// True once %globaltimer has passed the launch's deadline (a cached load
// and a special-register read: cheap enough for every few DFS steps).
__device__ __forceinline__ bool p_timed_out(const Ctl* c) {
    if (c->deadline == 0) return false;
    if (globaltimer_ns() > c->deadline) {
        atomicOr((unsigned*)&c->flags, (unsigned)KC_FLAG_TIMEOUT);
        return true;
    }
    return false;
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
    unsigned long long s = a + b;
    return (s < a || a == SAT || b == SAT) ? SAT : s;
}

__device__ __forceinline__ unsigned long long binom(const PivotParams& P, uint32_t a, int b) {
    if (b < 0 || (uint32_t)b > a || a >= P.bstride) return 0;
    return P.binom[(size_t)a * P.bstride + (uint32_t)b];
}

// per-vertex gain
__device__ __forceinline__ void pv_gain(const PivotParams& P, uint32_t vid, unsigned long long g) {
    if (g == 0) return;
    if (g == SAT) {
        atomicOr(&P.ctl->flags, (unsigned)KC_FLAG_VERTEX_OVERFLOW);
        return;
    }
    if (!in_bounds(P.ctl, vid, P.n, 101u)) return;
    unsigned long long old = atomicAdd(&P.pv[vid], g);
    if (old + g < old) atomicOr(&P.ctl->flags, (unsigned)KC_FLAG_VERTEX_OVERFLOW);
}

// Leaves of small (h, q) go to a per-block shared histogram (flushed at the
// end of the kernel), the rest straight to the global one.
static constexpr uint32_t LH = 16, LQ = 64;

__device__ __forceinline__ void leaf_store(const PivotParams& P, unsigned long long* hist, uint32_t h, uint32_t q,
                                           unsigned long long n) {
    if (h < LH && q < LQ) atomicAdd(&hist[h * LQ + q], n);
    else if (h < P.hq && q < P.hq) atomicAdd(&P.leaves[(size_t)h * P.hq + q], n);
    else atomicOr(&P.ctl->flags, (unsigned)KC_FLAG_INTERNAL);
}

// Run-length cache of leaves (lane 0 of a warp only).
struct LeafCache {
    unsigned long long* hist = nullptr;
    uint32_t h = 0, q = 0;
    unsigned long long n = 0;
    unsigned long long nodes = 0;  // tree nodes analysed by this warp
    __device__ __forceinline__ void flush(const PivotParams& P) {
        if (n) leaf_store(P, hist, h, q, n);
        n = 0;
    }
    __device__ __forceinline__ void add(const PivotParams& P, uint32_t hh, uint32_t qq) {
        if (n && hh == h && qq == q) {
            ++n;
            return;
        }
        flush(P);
        h = hh;
        q = qq;
        n = 1;
    }
};

// Warp-parallel analysis of the node with candidate set S (W words):
// returns cnt = |S|; kind 0 = empty, 1 = clique, 2 = internal with pivot p.
__device__ __forceinline__ int analyse(const uint32_t* S, const uint32_t* adj, uint32_t W, uint32_t& cnt,
                                       uint32_t& p) {
    const int lane = threadIdx.x & 31;
    if (W == 1) {
        const uint32_t s0 = S[0];
        cnt = __popc(s0);
        if (cnt <= 1) return (int)cnt;
        uint32_t best = 0, mind = 0xFFFFFFFFu;
        if ((s0 >> lane) & 1u) {
            const uint32_t dg = __popc(s0 & adj[lane]);
            best = (dg << 16) | (0xFFFFu - lane);
            mind = dg;
        }
        best = __reduce_max_sync(0xffffffffu, best);
        mind = __reduce_min_sync(0xffffffffu, mind);
        if (mind == cnt - 1) return 1;
        p = 0xFFFFu - (best & 0xFFFFu);
        return 2;
    }
    uint32_t c = 0;
    for (uint32_t w = lane; w < W; w += 32) c += __popc(S[w]);
    cnt = __reduce_add_sync(0xffffffffu, c);
    if (cnt == 0) return 0;
    if (cnt == 1) return 1;
    uint32_t best = 0, mind = 0xFFFFFFFFu;
    for (uint32_t w = 0; w < W; ++w) {
        const uint32_t bits = S[w];
        if (bits == 0) continue;
        if (lane < __popc(bits)) {
            const uint32_t u = (w << 5) + __fns(bits, 0, lane + 1);
            const uint32_t* au = adj + (size_t)u * W;
            uint32_t dg = 0;
            for (uint32_t x = 0; x < W; ++x) dg += __popc(S[x] & au[x]);
            best = max(best, (dg << 16) | (0xFFFFu - u));
            mind = min(mind, dg);
        }
    }
    best = __reduce_max_sync(0xffffffffu, best);
    mind = __reduce_min_sync(0xffffffffu, mind);
    if (mind == cnt - 1) return 1;
    p = 0xFFFFu - (best & 0xFFFFu);
    return 2;
}

// A walk's stack: level l (S_rem W | P_rem W | header HDR) in shared memory
// for l < ls, in global memory beyond.
struct Stk {
    uint32_t* s;
    uint32_t* g;
    uint32_t ls;
    uint32_t stride;
    __device__ __forceinline__ uint32_t* at(uint32_t l) const {
        return l < ls ? s + (size_t)l * stride : g + (size_t)(l - ls) * stride;
    }
};

// Per-warp scratch of a walk on one-word rows (a small root, or a node whose
// candidate set has been re-extracted into at most 32 vertices).
struct PNest {
    uint32_t cand[32];
    uint32_t adj[32];
    uint32_t S0[1];
    uint32_t pad[3];
    uint32_t stk[(PSMALL + 3) * (2 + HDR)];
    uint32_t pathbuf[64 + 1];  // vertices above an extracted walk (per-vertex mode)
    uint32_t pad2[3];
};

// Leaf (h, q) reached by choosing vertex vid (held or pivot); with PV, gains
// for vid and for the c clique members (pivots of the leaf) in S (if c > 0),
// and the leaf's contribution to the parent's subtree sums.
template <bool PV>
__device__ __forceinline__ void leaf(const PivotParams& P, LeafCache& lc, uint32_t h, uint32_t q, uint32_t vid,
                                     bool held, const uint32_t* S, uint32_t W, uint32_t c, const uint32_t* cand,
                                     unsigned long long& sumH, unsigned long long& sumP) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) lc.add(P, h, q);
    if (PV) {
        const int k = (int)P.pvk;
        const unsigned long long gH = binom(P, q, k - (int)h);
        const unsigned long long gP = q ? binom(P, q - 1, k - (int)h - 1) : 0ull;
        if (lane == 0) pv_gain(P, vid, held ? gH : gP);
        if (c && gP) {
            for (uint32_t w = 0; w < W; ++w) {
                uint32_t bits = S[w];
                if (lane < __popc(bits)) {
                    const uint32_t pos = (w << 5) + __fns(bits, 0, lane + 1);
                    if (in_bounds(P.ctl, pos, W == 1 ? 32u : P.dcap, 102u)) pv_gain(P, cand[pos], gP);
                }
            }
        }
        sumH = sat_add(sumH, gH);
        sumP = sat_add(sumP, gP);
    }
}

__device__ __forceinline__ void add_sums(uint32_t* hd, unsigned long long sH, unsigned long long sP) {
    unsigned long long pH = sat_add(((unsigned long long)hd[7] << 32) | hd[6], sH);
    unsigned long long pP = sat_add(((unsigned long long)hd[9] << 32) | hd[8], sP);
    hd[6] = (uint32_t)pH;
    hd[7] = (uint32_t)(pH >> 32);
    hd[8] = (uint32_t)pP;
    hd[9] = (uint32_t)(pP >> 32);
}

// ---------------------------------------------------------------------------
// Work stealing between the warps of a block, and between blocks through a
// global frame queue.  A frame is one level of a walk: S_rem (candidates),
// P_rem (branches not yet taken), h, q, the pivot and (per-vertex mode) the
// path of vertices above it.  A busy warp that sees idle warps (or, failing
// that, idle blocks) donates the upper half of P_rem of its shallowest frame
// with >= 2 branches: the thief's candidates exclude the donor's half (those
// branches come first in the iteration order), the donor keeps its half.
// ---------------------------------------------------------------------------
static constexpr int PQCAP = 16;
static constexpr int PPATH = 64;  // path entries a donated frame can carry
// A warp waiting for a frame of its block gives up after P_IDLE_NS, a block
// waiting for a frame of the global queue after P_GLOBAL_IDLE_NS (%globaltimer),
// and leaves the pool; donors finish their own work, so leaving is always
// safe (the count stays exact, only the help is lost).
static constexpr unsigned long long P_IDLE_NS = 2000000000ull;
static constexpr unsigned long long P_GLOBAL_IDLE_NS = 5000000000ull;

struct PStealShared {
    unsigned idle, active, queued;
    unsigned state[PQCAP];
};

__device__ __forceinline__ unsigned pvld(const unsigned* p) { return *(const volatile unsigned*)p; }

// Frame slot layout (local and global queues alike):
//   [0] kind (0: rows of the root's bitmap, W words; 1: one-word rows carried
//       in the slot), [1] root slot (kind 0), [2..5] h, q, pivot, npath,
//   [6, 6 + PPATH) path, then kind 0: S (W0) | P (W0);
//   kind 1: S | P | adj (32) | vertex ids (32).
static constexpr uint32_t SLOT_HDR = 6 + PPATH;
__host__ __device__ __forceinline__ uint32_t pq_stride(uint32_t W0) {
    return SLOT_HDR + (2 * W0 > 66 ? 2 * W0 : 66);
}

// Credit the vertices of a base path with a subtree's sums (lanes over entries).
__device__ __forceinline__ void credit_path(const PivotParams& P, const uint32_t* path, uint32_t npath,
                                            unsigned long long sH, unsigned long long sP) {
    const int lane = threadIdx.x & 31;
    for (uint32_t i = lane; i < npath; i += 32) {
        const uint32_t e = path[i];
        pv_gain(P, e & 0x7FFFFFFFu, (e >> 31) ? sH : sP);
    }
}

template <bool PV, bool WIDE>
__device__ void walk_levels(const PivotParams& P, const uint32_t* adj, uint32_t W, const uint32_t* cand, Stk stk,
                            uint32_t lvl_cap, LeafCache& lc, const uint32_t* path, uint32_t npath, PStealShared* ss,
                            uint32_t* qwords, uint32_t W0, uint32_t root_slot, PNest* nest, unsigned long long& topH,
                            unsigned long long& topP, const uint32_t* outer = nullptr, uint32_t nouter = 0);

// Walk the subtree of the start node (candidates S0, h0, q0) reached by
// choosing vertex vid0 (held0).  topH/topP: the node's subtree sums
// (per-vertex mode) for the caller to credit the vertices above it.
template <bool PV, bool WIDE>
__device__ void warp_walk(const PivotParams& P, const uint32_t* adj, uint32_t W, const uint32_t* cand, Stk stk,
                          uint32_t lvl_cap, const uint32_t* S0, uint32_t h0, uint32_t q0, uint32_t vid0, bool held0,
                          LeafCache& lc, PStealShared* ss, uint32_t* qwords, uint32_t W0, uint32_t root_slot,
                          PNest* nest, unsigned long long& topH, unsigned long long& topP,
                          const uint32_t* outer = nullptr, uint32_t nouter = 0) {
    const int lane = threadIdx.x & 31;
    topH = topP = 0;
    uint32_t* L0 = stk.at(0);
    for (uint32_t w = lane; w < W; w += 32) L0[w] = S0[w];
    __syncwarp();
    uint32_t cnt, p = 0;
    int kind = analyse(L0, adj, W, cnt, p);
    if (lane == 0) ++lc.nodes;
    if (kind != 2) {
        const uint32_t c = kind == 1 ? cnt : 0;
        leaf<PV>(P, lc, h0, q0 + c, vid0, held0, L0, W, c, cand, topH, topP);
        return;
    }
    const uint32_t* ap = adj + (size_t)p * W;
    for (uint32_t w = lane; w < W; w += 32) L0[W + w] = L0[w] & ~ap[w];
    if (lane == 0) {
        uint32_t* hd = L0 + 2 * W;
        hd[0] = h0; hd[1] = q0; hd[2] = p; hd[3] = vid0; hd[4] = held0;
        hd[6] = hd[7] = hd[8] = hd[9] = 0;
    }
    __syncwarp();
    // level 0 credits just its own vertex; the outer path (the vertices above,
    // credited by the caller) only travels with donated frames
    const uint32_t path0 = vid0 | (held0 ? 0x80000000u : 0u);
    walk_levels<PV, WIDE>(P, adj, W, cand, stk, lvl_cap, lc, &path0, 1, ss, qwords, W0, root_slot, nest, topH, topP,
                          outer, nouter);
}

// Re-extract the candidate set S (cnt <= 32 members, W words) into a one-word
// sub-graph in nest and walk it from (h, q) reached by vid (held).
template <bool PV>
__device__ void walk_extracted(const PivotParams& P, const uint32_t* adj, uint32_t W, const uint32_t* cand,
                               const uint32_t* S, uint32_t cnt, uint32_t h, uint32_t q, uint32_t vid, bool held,
                               LeafCache& lc, PNest* nest, const uint32_t* path, uint32_t npath, PStealShared* ss,
                               uint32_t* qwords, uint32_t W0, unsigned long long& sH, unsigned long long& sP) {
    const int lane = threadIdx.x & 31;
    uint32_t mine = NONE, base = 0;
    for (uint32_t w = 0; w < W; ++w) {
        const uint32_t bits = S[w], c = __popc(bits);
        if ((uint32_t)lane >= base && (uint32_t)lane < base + c) mine = (w << 5) + __fns(bits, 0, lane - base + 1);
        base += c;
    }
    uint32_t row = 0;
    if (mine != NONE) {
        const uint32_t* am = adj + (size_t)mine * W;
        uint32_t b = 0;
        for (uint32_t w = 0; w < W; ++w) {
            const uint32_t sw = S[w];
            uint32_t bits = am[w] & sw;
            while (bits) {
                const uint32_t pos = __ffs(bits) - 1;
                bits &= bits - 1;
                row |= 1u << (b + __popc(sw & ((1u << pos) - 1u)));
            }
            b += __popc(sw);
        }
    }
    __syncwarp();
    nest->adj[lane] = row;
    nest->cand[lane] = mine != NONE ? cand[mine] : 0;
    if (lane == 0) nest->S0[0] = cnt == 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u);
    __syncwarp();
    Stk small{nest->stk, nullptr, PSMALL + 3, 2 + HDR};
    warp_walk<PV, false>(P, nest->adj, 1, nest->cand, small, PSMALL + 3, nest->S0, h, q, vid, held, lc, ss, qwords,
                         W0, 0, nullptr, sH, sP, path, npath);
}

// The DFS from a level 0 already in stk (S_rem, P_rem, header).  path/npath:
// the vertices above level 0's children (level 0's own vertex last), each
// with its held flag in bit 31.  topH/topP: level 0's subtree sums.
template <bool PV, bool WIDE>
__device__ void walk_levels(const PivotParams& P, const uint32_t* adj, uint32_t W, const uint32_t* cand, Stk stk,
                            uint32_t lvl_cap, LeafCache& lc, const uint32_t* path, uint32_t npath, PStealShared* ss,
                            uint32_t* qwords, uint32_t W0, uint32_t root_slot, PNest* nest, unsigned long long& topH,
                            unsigned long long& topP, const uint32_t* outer, uint32_t nouter) {
    const int lane = threadIdx.x & 31;
    const uint32_t k = P.kfix;
    PWorkCtl* wc = reinterpret_cast<PWorkCtl*>(P.ctl + 1);
    topH = topP = 0;
    int l = 0;
    uint32_t steps = 0;
    for (;;) {
        if ((++steps & 15u) == 0) {
            {
                int to = lane == 0 ? (int)p_timed_out(P.ctl) : 0;
                if (__shfl_sync(0xffffffffu, to, 0)) break;
            }
            // 1: an idle warp of this block; 2: an idle block anywhere
            int want = 0;
            if (lane == 0) {
                if (ss && pvld(&ss->idle) > 0 && pvld(&ss->queued) < PQCAP) want = 1;
                else if (P.gq_cap && pvld(&wc->g_idle) > 0 && pvld(&wc->g_queued) < P.gq_cap) want = 2;
            }
            want = __shfl_sync(0xffffffffu, want, 0);
            if (want) {
                for (int lv = 0; lv <= l; ++lv) {
                    if (PV && nouter + npath + lv > PPATH) break;
                    uint32_t* Lv = stk.at(lv);
                    uint32_t c = 0;
                    for (uint32_t w = lane; w < W; w += 32) c += __popc(Lv[W + w]);
                    c = __reduce_add_sync(0xffffffffu, c);
                    if (c < 2) continue;
                    uint32_t q = NONE, split = NONE;
                    if (lane == 0) {
                        uint32_t m = c / 2;  // keep the first m branches
                        for (uint32_t w = 0; w < W && split == NONE; ++w) {
                            const uint32_t x = Lv[W + w], pc = __popc(x);
                            if (m < pc) split = (w << 5) + __fns(x, 0, m + 1);
                            else m -= pc;
                        }
                        unsigned* st = want == 1 ? ss->state : P.gq_state;
                        const uint32_t cap = want == 1 ? PQCAP : P.gq_cap;
                        for (uint32_t x = 0; x < cap; ++x)
                            if (pvld(&st[x]) == 0 && atomicCAS(&st[x], 0u, 1u) == 0u) {
                                q = x;
                                break;
                            }
                    }
                    q = __shfl_sync(0xffffffffu, q, 0);
                    split = __shfl_sync(0xffffffffu, split, 0);
                    if (q == NONE || split == NONE) {
                        if (lane == 0 && q != NONE) atomicExch(want == 1 ? &ss->state[q] : &P.gq_state[q], 0u);
                        break;
                    }
                    uint32_t* dst = want == 1 ? qwords + (size_t)q * pq_stride(W0) : P.gq + (size_t)q * P.gq_stride;
                    const uint32_t* hv = Lv + 2 * W;
                    uint32_t* dS = dst + SLOT_HDR;
                    uint32_t* dP = dst + SLOT_HDR + (WIDE ? W0 : 1);
                    for (uint32_t w = lane; w < W; w += 32) {
                        const uint32_t bw = w << 5;
                        const uint32_t hi_mask = bw + 31 < split ? 0u : (bw >= split ? 0xFFFFFFFFu
                                                                                    : 0xFFFFFFFFu << (split - bw));
                        const uint32_t pr = Lv[W + w];
                        dS[w] = Lv[w] & ~(pr & ~hi_mask);  // without the donor's branches
                        dP[w] = pr & hi_mask;               // the thief's branches
                    }
                    if (!WIDE) {  // the one-word sub-graph travels with the frame
                        dst[SLOT_HDR + 2 + lane] = adj[lane];
                        dst[SLOT_HDR + 34 + lane] = cand[lane];
                    }
                    if (lane == 0) {
                        dst[0] = WIDE ? 0u : 1u;
                        dst[1] = root_slot;
                        dst[2] = hv[0];
                        dst[3] = hv[1];
                        dst[4] = hv[2];
                        dst[5] = PV ? nouter + npath + lv : 0;
                    }
                    if (PV) {
                        uint32_t* dp = dst + 6;
                        for (uint32_t i = lane; i < nouter; i += 32) dp[i] = outer[i];
                        for (uint32_t i = lane; i < npath; i += 32) dp[nouter + i] = path[i];
                        for (int i = 1 + lane; i <= lv; i += 32) {
                            const uint32_t* hi = stk.at(i) + 2 * W;
                            dp[nouter + npath + i - 1] = hi[3] | (hi[4] ? 0x80000000u : 0u);
                        }
                    }
                    __syncwarp();
                    for (uint32_t w = lane; w < W; w += 32) {  // the donor keeps the lower half
                        const uint32_t bw = w << 5;
                        const uint32_t lo_mask = bw + 31 < split ? 0xFFFFFFFFu
                                                                 : (bw >= split ? 0u : ~(0xFFFFFFFFu << (split - bw)));
                        Lv[W + w] &= lo_mask;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        if (want == 1) {
                            __threadfence_block();
                            atomicExch(&ss->state[q], 2u);
                            atomicAdd(&ss->queued, 1u);
                        } else {
                            __threadfence();
                            atomicExch(&P.gq_state[q], 2u);
                            atomicAdd(&wc->g_queued, 1u);
                        }
                    }
                    break;
                }
            }
        }
        uint32_t* Lc = stk.at(l);
        uint32_t* hd = Lc + 2 * W;
        const uint32_t x = next_bit(Lc + W, 0, W - 1);
        if (x == NONE) {
            // subtree of level l done
            if (PV) {
                unsigned long long sH = ((unsigned long long)hd[7] << 32) | hd[6];
                unsigned long long sP = ((unsigned long long)hd[9] << 32) | hd[8];
                if (l == 0) {
                    credit_path(P, path, npath, sH, sP);
                    topH = sH;
                    topP = sP;
                } else {
                    if (lane == 0) {
                        pv_gain(P, hd[3], hd[4] ? sH : sP);
                        add_sums(stk.at(l - 1) + 2 * W, sH, sP);
                    }
                    __syncwarp();
                }
            }
            if (l == 0) break;
            --l;
            continue;
        }
        const uint32_t h = hd[0], q = hd[1], piv = hd[2];
        __syncwarp();
        if (lane == 0) Lc[W + (x >> 5)] &= ~(1u << (x & 31));  // visited
        if ((uint32_t)l + 1 >= lvl_cap) {  // cannot happen: depth <= clique number <= |C| + 1
            if (lane == 0) atomicOr(&P.ctl->flags, (unsigned)KC_FLAG_INTERNAL);
            break;
        }
        // child candidates: S_rem ∩ N(x); x then leaves S_rem for later siblings
        uint32_t* Ln = stk.at(l + 1);
        const uint32_t* ax = adj + (size_t)x * W;
        for (uint32_t w = lane; w < W; w += 32) Ln[w] = Lc[w] & ax[w];
        __syncwarp();
        if (lane == 0) Lc[x >> 5] &= ~(1u << (x & 31));
        const bool xheld = x != piv;
        const uint32_t h2 = h + (xheld ? 1u : 0u), q2 = q + (xheld ? 0u : 1u);
        if (k && h2 > k) {
            __syncwarp();
            continue;
        }
        uint32_t cnt2 = 0, p2 = 0;
        if (WIDE && W > 1) {
            uint32_t c = 0;
            for (uint32_t w = lane; w < W; w += 32) c += __popc(Ln[w]);
            cnt2 = __reduce_add_sync(0xffffffffu, c);
            if (k && h2 + q2 + cnt2 < k) {
                __syncwarp();
                continue;
            }
            if (cnt2 <= 32) {
                // few candidates left: walk this child on one-word rows; for a frame
                // it donates, the vertices above it are this walk's path plus levels 1..l
                uint32_t nout = 0;
                if (PV) {
                    uint32_t* ob = nest->pathbuf;
                    for (uint32_t i = lane; i < nouter && i < PPATH; i += 32) ob[i] = outer[i];
                    for (uint32_t i = lane; i < npath && nouter + i < PPATH; i += 32) ob[nouter + i] = path[i];
                    for (int i = 1 + lane; i <= l && nouter + npath + i - 1 < PPATH; i += 32) {
                        const uint32_t* hi = stk.at(i) + 2 * W;
                        ob[nouter + npath + i - 1] = hi[3] | (hi[4] ? 0x80000000u : 0u);
                    }
                    nout = min(nouter + npath + (uint32_t)l, (uint32_t)PPATH + 1);
                    __syncwarp();
                }
                unsigned long long sH = 0, sP = 0;
                walk_extracted<PV>(P, adj, W, cand, Ln, cnt2, h2, q2, cand[x], xheld, lc, nest, nest->pathbuf, nout,
                                   ss, qwords, W0, sH, sP);
                if (PV && lane == 0) add_sums(hd, sH, sP);
                __syncwarp();
                continue;
            }
        }
        int kind2 = analyse(Ln, adj, W, cnt2, p2);
        if (lane == 0) ++lc.nodes;
        if (k && h2 + q2 + cnt2 < k) {
            __syncwarp();
            continue;
        }
        if (kind2 != 2) {
            const uint32_t c = kind2 == 1 ? cnt2 : 0;
            unsigned long long sH = 0, sP = 0;
            leaf<PV>(P, lc, h2, q2 + c, cand[x], xheld, Ln, W, c, cand, sH, sP);
            if (PV && lane == 0) add_sums(hd, sH, sP);
            __syncwarp();
            continue;
        }
        const uint32_t* ap = adj + (size_t)p2 * W;
        for (uint32_t w = lane; w < W; w += 32) Ln[W + w] = Ln[w] & ~ap[w];
        if (lane == 0) {
            uint32_t* nh = Ln + 2 * W;
            nh[0] = h2; nh[1] = q2; nh[2] = p2; nh[3] = cand[x]; nh[4] = xheld;
            nh[6] = nh[7] = nh[8] = nh[9] = 0;
        }
        __syncwarp();
        ++l;
    }
}

// The per-warp pieces of the block layout a taken frame needs.
struct PLayoutLite {
    uint32_t* qwords;
    uint32_t* wpath;
    PNest* nest;
    Stk stk;
};

// Copy a donated frame (slot src) into this warp's walk state: kind 0 into
// level 0 of the wide stack, kind 1 into the one-word scratch nest.  The path
// goes to path.  Returns (kind << 16) | npath.
__device__ uint32_t take_frame(const uint32_t* src, uint32_t W0, uint32_t W, Stk stk, PNest* nest, uint32_t* path) {
    const int lane = threadIdx.x & 31;
    const uint32_t kind = src[0], np = src[5];
    for (uint32_t i = lane; i < np; i += 32) path[i] = src[6 + i];
    uint32_t* L0;
    uint32_t w1;
    if (kind == 0) {
        L0 = stk.at(0);
        w1 = W;
        for (uint32_t w = lane; w < W; w += 32) {
            L0[w] = src[SLOT_HDR + w];
            L0[W + w] = src[SLOT_HDR + W0 + w];
        }
    } else {
        L0 = nest->stk;
        w1 = 1;
        nest->adj[lane] = src[SLOT_HDR + 2 + lane];
        nest->cand[lane] = src[SLOT_HDR + 34 + lane];
        if (lane == 0) {
            L0[0] = src[SLOT_HDR];
            L0[1] = src[SLOT_HDR + 1];
        }
    }
    if (lane == 0) {
        uint32_t* hd = L0 + 2 * w1;
        hd[0] = src[2];
        hd[1] = src[3];
        hd[2] = src[4];
        hd[3] = NONE;
        hd[4] = 0;
        hd[6] = hd[7] = hd[8] = hd[9] = 0;
    }
    __syncwarp();
    return (kind << 16) | np;
}

// A warp out of branches: take a frame from the block's queue, or learn that
// the session is over.  Returns 1 + ((kind << 16) | npath) when a frame was
// taken, 0 otherwise.
__device__ uint32_t p_steal_or_finish(const PivotParams& P, PStealShared* ss, uint32_t* qwords, uint32_t W0,
                                      uint32_t W, Stk stk, PNest* nest, uint32_t* path) {
    const int lane = threadIdx.x & 31;
    uint32_t q = NONE;
    if (lane == 0) {
        int done = 0;
        atomicAdd(&ss->idle, 1u);
        const unsigned long long t0 = globaltimer_ns();
        for (uint32_t it = 0;; ++it) {
            if ((it & 255u) == 255u && globaltimer_ns() - t0 > P_IDLE_NS) break;
            if (pvld(&ss->queued) > 0) {
                atomicSub(&ss->idle, 1u);
                for (uint32_t x = 0; x < PQCAP; ++x)
                    if (pvld(&ss->state[x]) == 2u && atomicCAS(&ss->state[x], 2u, 3u) == 2u) {
                        q = x;
                        break;
                    }
                if (q != NONE) {
                    atomicSub(&ss->queued, 1u);
                    break;
                }
                atomicAdd(&ss->idle, 1u);
            }
            if (pvld(&ss->idle) == pvld(&ss->active) && pvld(&ss->queued) == 0) {
                done = 1;
                break;
            }
            if ((it & 1023u) == 1023u && p_timed_out(P.ctl)) {
                atomicSub(&ss->idle, 1u);
                atomicSub(&ss->active, 1u);
                done = 1;
                break;
            }
            __nanosleep(256);
        }
        if (q == NONE && !done) {  // waited long enough: leave the pool (donors finish their own work)
            atomicSub(&ss->idle, 1u);
            atomicSub(&ss->active, 1u);
        }
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q == NONE) return 0;
    __threadfence_block();
    const uint32_t r = take_frame(qwords + (size_t)q * pq_stride(W0), W0, W, stk, nest, path);
    if (lane == 0) atomicExch(&ss->state[q], 0u);
    return r + 1;
}

// Walk a taken frame (kind 0 on the block's root bitmap, kind 1 on its own
// one-word sub-graph); the frame's path already holds every vertex above it.
template <bool PV>
__device__ void walk_taken(const PivotParams& P, uint32_t r, const uint32_t* adj, uint32_t W, const uint32_t* cand,
                           const PLayoutLite& L, LeafCache& lc, PStealShared* ss, uint32_t root_slot) {
    const uint32_t kind = r >> 16, np = r & 0xFFFFu;
    unsigned long long sH = 0, sP = 0;
    if (kind == 0) {
        walk_levels<PV, true>(P, adj, W, cand, L.stk, P.lvl_cap, lc, L.wpath, np, ss, L.qwords, P.wcap, root_slot,
                              L.nest, sH, sP);
    } else {
        Stk small{L.nest->stk, nullptr, PSMALL + 3, 2 + HDR};
        walk_levels<PV, false>(P, L.nest->adj, 1, L.nest->cand, small, PSMALL + 3, lc, L.wpath, np, ss, L.qwords,
                               P.wcap, 0, nullptr, sH, sP);
    }
}

// Undirected adjacency of the candidates: OR every row with its transpose.
template <int NT>
__device__ void symmetrise(uint32_t* adj, uint32_t d, uint32_t W) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t i = warp; i < d; i += NT / 32) {
        const uint32_t* ri = adj + (size_t)i * W;
        for (uint32_t w = lane; w < W; w += 32) {
            uint32_t bits = ri[w] & ((w << 5) + 31 > i ? 0xFFFFFFFFu : 0u);
            while (bits) {
                const uint32_t j = (w << 5) + (__ffs(bits) - 1);
                bits &= bits - 1;
                if (j > i) atomicOr(&adj[(size_t)j * W + (i >> 5)], 1u << (i & 31));
            }
        }
    }
    __syncthreads();
}

struct PBlockShared {
    uint32_t slot;
    uint32_t pivot;
    uint32_t ntask;
    uint32_t kind;
    uint32_t mind;
    unsigned long long best;
};

// Shared-memory layout of the block phases (word offsets from psmem).
struct PLayout {
    uint32_t* cand;
    uint32_t* adj;
    uint32_t* pre;
    uint32_t* Sx;      // this warp's start set
    uint32_t* qwords;  // donated frames
    uint32_t* wpath;   // this warp's taken-frame path
    PNest* nest;       // this warp's one-word-row scratch
    Stk stk;           // this warp's wide stack
};

__device__ __forceinline__ PLayoutLite lite(const PLayout& L) { return PLayoutLite{L.qwords, L.wpath, L.nest, L.stk}; }

__device__ __forceinline__ PLayout layout(const PivotParams& P, uint32_t* smem) {
    const int warp = threadIdx.x >> 5;
    const uint32_t D0 = (P.dcap + 31) & ~31u;
    PLayout L;
    L.cand = smem;
    uint32_t* p = smem + D0;
    if (P.adj_in_smem) {
        L.adj = p;
        p += (size_t)P.dcap * P.wcap;
    } else {
        L.adj = P.gadj + (size_t)blockIdx.x * P.gadj_words;
    }
    L.pre = p;
    p += P.wcap + 32;
    L.Sx = p + (size_t)warp * P.wcap;
    p += (size_t)PW * P.wcap;
    L.qwords = p;
    p += (size_t)PQCAP * pq_stride(P.wcap);
    L.wpath = p + (size_t)warp * PPATH;
    p += (size_t)PW * PPATH;
    L.nest = reinterpret_cast<PNest*>(p) + warp;
    p += (size_t)PW * (sizeof(PNest) / 4);
    const uint32_t stride = 2 * P.wcap + HDR;
    L.stk.s = p + (size_t)warp * P.lvl_smem * stride;
    L.stk.g = P.gstack + ((size_t)blockIdx.x * PW + warp) * P.gstack_words;
    L.stk.ls = P.lvl_smem;
    L.stk.stride = stride;
    return L;
}

__device__ __forceinline__ void reset_session(PStealShared& ss) {
    if (threadIdx.x == 0) {
        ss.idle = 0;
        ss.active = PW;
        ss.queued = 0;
        for (int x = 0; x < PQCAP; ++x) ss.state[x] = 0;
    }
    __syncthreads();
}

template <bool PV>
__device__ void pivot_block_phase(const PivotParams& P, uint32_t* smem, PBlockShared& sh, PStealShared& ss,
                                  LeafCache& lc) {
    PWorkCtl* wc = reinterpret_cast<PWorkCtl*>(P.ctl + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const PLayout L = layout(P, smem);
    uint32_t* cand = L.cand;
    uint32_t* adj = L.adj;
    uint32_t* pre = L.pre;
    int phase = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t s = NONE;
            if (!p_timed_out(P.ctl)) {
                if (phase == 0) {
                    s = atomicAdd(&wc->root_cursor, 1u);
                    if (s >= P.n_big) {
                        phase = 1;
                        s = NONE;
                    }
                }
                if (phase == 1) {
                    uint32_t lo = atomicAdd(&wc->help_lo, 0u);
                    for (uint32_t probes = 0; lo < P.n_big && probes < 4096; ++lo, ++probes) {
                        // a root is worth joining while >= 2 branches may be unclaimed; the
                        // branch count is unknown until its pivot is chosen, so use d
                        const uint32_t u = P.roots[lo];
                        const uint32_t d = P.rp[u + 1] - P.rp[u];
                        const uint32_t taken = atomicAdd(&P.task_next[lo], 0u);
                        if (taken + 2 <= d && taken < 0x7FFFFFFFu) {
                            s = lo;
                            break;
                        }
                        atomicMax(&wc->help_lo, lo + 1);
                    }
                }
            }
            sh.slot = s;
            sh.best = 0;
            sh.mind = 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t s = sh.slot;
        if (s == NONE) break;
        const uint32_t u = P.roots[s];
        const uint32_t b = P.rp[u], d = P.rp[u + 1] - b;
        for (uint32_t i = threadIdx.x; i < d; i += PB) cand[i] = P.col[b + i];
        __syncthreads();
        const uint32_t W = (d + 31) >> 5;
        build_bitmap<PB>(P.rp, P.col, cand, d, W, adj);
        symmetrise<PB>(adj, d, W);
        // root pivot: the candidate with the most neighbours (all of C is the
        // root node's candidate set); ties to the lowest index
        {
            unsigned long long best = 0;
            uint32_t mind = 0xFFFFFFFFu;
            for (uint32_t x = threadIdx.x; x < d; x += PB) {
                const uint32_t* ax = adj + (size_t)x * W;
                uint32_t dg = 0;
                for (uint32_t w = 0; w < W; ++w) dg += __popc(ax[w]);
                best = max(best, ((unsigned long long)dg << 32) | (0xFFFFFFFFu - x));
                mind = min(mind, dg);
            }
            for (int o = 16; o > 0; o >>= 1) {
                best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
                mind = min(mind, __shfl_xor_sync(0xffffffffu, mind, o));
            }
            if (lane == 0) {
                atomicMax(&sh.best, best);
                atomicMin(&sh.mind, mind);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                sh.pivot = 0xFFFFFFFFu - (uint32_t)(sh.best & 0xFFFFFFFFu);
                sh.kind = (sh.mind == d - 1) ? 1u : 2u;
            }
            __syncthreads();
        }
        if (sh.kind == 1) {
            // the whole candidate set is a clique: one leaf (1, d), taken by one block
            if (threadIdx.x == 0 && atomicCAS(&P.task_next[s], 0u, 0x80000000u) == 0u) {
                if (!(P.kfix && 1 + d < P.kfix)) {
                    lc.add(P, 1, d);
                    if (PV) {
                        const int k = (int)P.pvk;
                        pv_gain(P, u, binom(P, d, k - 1));
                        const unsigned long long gP = binom(P, d - 1, k - 2);
                        for (uint32_t i = 0; i < d; ++i) pv_gain(P, cand[i], gP);
                    }
                }
            }
            __syncthreads();
            continue;
        }
        const uint32_t piv = sh.pivot;
        const uint32_t* apv = adj + (size_t)piv * W;
        // branch set of the root: C \ N(p); prefix popcounts of its words
        if (warp == 0) {
            uint32_t carry = 0;
            for (uint32_t w0 = 0; w0 < W; w0 += 32) {
                const uint32_t w = w0 + lane;
                uint32_t pr = 0;
                if (w < W) {
                    const uint32_t valid = (w == W - 1 && (d & 31)) ? ((1u << (d & 31)) - 1u) : 0xFFFFFFFFu;
                    pr = ~apv[w] & valid;
                }
                const uint32_t c = __popc(pr);
                uint32_t incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (w < W) pre[w] = carry + incl - c;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) {
                pre[W] = carry;
                sh.ntask = carry;
            }
        }
        __syncthreads();
        const uint32_t ntask = sh.ntask;
        reset_session(ss);
        for (;;) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(&P.task_next[s], 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= ntask) {
                // every branch is claimed: keep other blocks from joining this root
                if (lane == 0) atomicMax(&P.task_next[s], 0x7FFFFFFFu);
                break;
            }
            // the t-th member x of the branch set
            uint32_t lo = 0, hi = W;  // last word with pre[w] <= t
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (pre[mid] <= t) lo = mid; else hi = mid;
            }
            const uint32_t valid_lo = (lo == W - 1 && (d & 31)) ? ((1u << (d & 31)) - 1u) : 0xFFFFFFFFu;
            const uint32_t prw = ~apv[lo] & valid_lo;
            const uint32_t x = (lo << 5) + __fns(prw, 0, t - pre[lo] + 1);
            const uint32_t* ax = adj + (size_t)x * W;
            // S_x = C ∩ N(x) minus the branch members before x
            for (uint32_t w = lane; w < W; w += 32) {
                const uint32_t valid = (w == W - 1 && (d & 31)) ? ((1u << (d & 31)) - 1u) : 0xFFFFFFFFu;
                const uint32_t prw2 = ~apv[w] & valid;
                uint32_t before = 0;
                if (w < (x >> 5)) before = prw2;
                else if (w == (x >> 5)) before = prw2 & ((1u << (x & 31)) - 1u);
                L.Sx[w] = ax[w] & valid & ~before;
            }
            __syncwarp();
            const bool xheld = x != piv;
            const uint32_t h0 = 1 + (xheld ? 1u : 0u), q0 = xheld ? 0u : 1u;
            if (P.kfix && h0 > P.kfix) continue;
            unsigned long long sH = 0, sP = 0;
            const uint32_t root_entry = u | 0x80000000u;  // the root is held in every clique below it
            warp_walk<PV, true>(P, adj, W, cand, L.stk, P.lvl_cap, L.Sx, h0, q0, cand[x], xheld, lc, &ss, L.qwords,
                                P.wcap, s, L.nest, sH, sP, &root_entry, 1);
            if (PV && lane == 0) pv_gain(P, u, sH);
            if (lane == 0 && p_timed_out(P.ctl)) t = NONE;
            if (__shfl_sync(0xffffffffu, t, 0) == NONE) break;
        }
        for (;;) {
            const uint32_t got = p_steal_or_finish(P, &ss, L.qwords, P.wcap, W, L.stk, L.nest, L.wpath);
            if (!got) break;
            walk_taken<PV>(P, got - 1, adj, W, cand, lite(L), lc, &ss, s);
        }
        __syncthreads();
    }
}

// Warp mode: one warp per small root, rows of one word.
template <bool PV>
__device__ void pivot_warp_phase(const PivotParams& P, PNest& ws, LeafCache& lc) {
    PWorkCtl* wc = reinterpret_cast<PWorkCtl*>(P.ctl + 1);
    const int lane = threadIdx.x & 31;
    uint32_t iter = 0;
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) {
            i = P.n_big + atomicAdd(&wc->small_cursor, 1u);
            if ((++iter & 63u) == 0 && p_timed_out(P.ctl)) i = NONE;
        }
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= P.n_work) break;
        const uint32_t u = P.roots[i];
        const uint32_t b = P.rp[u];
        const uint32_t d = P.rp[u + 1] - b;
        if (lane < (int)d) ws.cand[lane] = P.col[b + lane];
        __syncwarp();
        const uint32_t last = ws.cand[d - 1];
        uint32_t myrow = 0;
        uint32_t rb = 0, re = 0;
        if (lane < (int)d) {
            rb = __ldg(P.rp + ws.cand[lane]);
            re = __ldg(P.rp + ws.cand[lane] + 1);
        }
        for (uint32_t r = 0; r < d; ++r) {
            const uint32_t xb = __shfl_sync(0xffffffffu, rb, r), xe = __shfl_sync(0xffffffffu, re, r);
            uint32_t bits = 0;
            scan_row(P.col, xb, xe, last, lane, [&](uint32_t y) {
                const uint32_t pos = find_sorted(ws.cand, r + 1, d, y);
                if (pos != NONE) bits |= 1u << pos;
            });
            bits = __reduce_or_sync(0xffffffffu, bits);
            if (lane == (int)r) myrow = bits;
        }
        // undirected row of candidate `lane`: its out-row plus the rows that name it
        uint32_t colbits = 0;
        for (uint32_t r = 0; r < d; ++r) {
            uint32_t rr = __shfl_sync(0xffffffffu, myrow, r);
            if ((rr >> lane) & 1u) colbits |= 1u << r;
        }
        ws.adj[lane] = lane < (int)d ? (myrow | colbits) : 0u;
        if (lane == 0) ws.S0[0] = d == 32 ? 0xFFFFFFFFu : ((1u << d) - 1u);
        __syncwarp();
        unsigned long long sH = 0, sP = 0;
        Stk small{ws.stk, nullptr, PSMALL + 3, 2 + HDR};
        warp_walk<PV, false>(P, ws.adj, 1, ws.cand, small, PSMALL + 3, ws.S0, 1, 0, u, true, lc, nullptr, nullptr,
                             P.wcap, 0, nullptr, sH, sP);
        __syncwarp();
    }
}

// Blocks with nothing left of their own serve the global frame queue: take a
// frame, rebuild that root's bitmap, and walk the frame with the block's warps
// (warp 0 starts it, the others steal from it).  The wait is bounded; a block
// that gives up leaves the pool, and donors finish their own work.
__device__ uint32_t global_take(const PivotParams& P) {
    PWorkCtl* wc = reinterpret_cast<PWorkCtl*>(P.ctl + 1);
    atomicAdd(&wc->g_idle, 1u);
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t it = 0;; ++it) {
        if ((it & 255u) == 255u && globaltimer_ns() - t0 > P_GLOBAL_IDLE_NS) break;
        if (pvld(&wc->g_queued) > 0) {
            atomicSub(&wc->g_idle, 1u);
            for (uint32_t x = 0; x < P.gq_cap; ++x)
                if (pvld(&P.gq_state[x]) == 2u && atomicCAS(&P.gq_state[x], 2u, 3u) == 2u) {
                    atomicSub(&wc->g_queued, 1u);
                    __threadfence();
                    return x;
                }
            atomicAdd(&wc->g_idle, 1u);
        }
        if (pvld(&wc->g_idle) == pvld(&wc->g_active) && pvld(&wc->g_queued) == 0) return NONE;
        if ((it & 1023u) == 1023u && p_timed_out(P.ctl)) break;
        __nanosleep(512);
    }
    atomicSub(&wc->g_idle, 1u);
    atomicSub(&wc->g_active, 1u);
    return NONE;
}

template <bool PV>
__device__ void pivot_global_phase(const PivotParams& P, uint32_t* smem, PBlockShared& sh, PStealShared& ss,
                                   LeafCache& lc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const PLayout L = layout(P, smem);
    uint32_t* cand = L.cand;
    uint32_t* adj = L.adj;
    for (;;) {
        if (threadIdx.x == 0) sh.slot = global_take(P);
        __syncthreads();
        const uint32_t q = sh.slot;
        if (q == NONE) break;
        const uint32_t* g = P.gq + (size_t)q * P.gq_stride;
        const uint32_t kind = g[0], s = g[1];
        uint32_t W = 1;
        if (kind == 0) {  // a frame on a root's bitmap: rebuild that bitmap here
            const uint32_t u = P.roots[s];
            const uint32_t b = P.rp[u], d = P.rp[u + 1] - b;
            for (uint32_t i = threadIdx.x; i < d; i += PB) cand[i] = P.col[b + i];
            __syncthreads();
            W = (d + 31) >> 5;
            build_bitmap<PB>(P.rp, P.col, cand, d, W, adj);
            symmetrise<PB>(adj, d, W);
        }
        reset_session(ss);
        if (warp == 0) {
            const uint32_t r = take_frame(g, P.wcap, W, L.stk, L.nest, L.wpath);
            if (lane == 0) atomicExch(&P.gq_state[q], 0u);
            walk_taken<PV>(P, r, adj, W, cand, lite(L), lc, &ss, s);
        }
        for (;;) {
            const uint32_t got = p_steal_or_finish(P, &ss, L.qwords, P.wcap, W, L.stk, L.nest, L.wpath);
            if (!got) break;
            walk_taken<PV>(P, got - 1, adj, W, cand, lite(L), lc, &ss, s);
        }
        __syncthreads();
    }
}

template <bool PV>
__global__ void __launch_bounds__(PB) k_count_pivot(const PivotParams P) {
    extern __shared__ __align__(16) uint32_t psmem[];
    __shared__ PBlockShared sh;
    __shared__ PStealShared ss;
    __shared__ unsigned long long s_hist[LH * LQ];
    for (uint32_t i = threadIdx.x; i < LH * LQ; i += PB) s_hist[i] = 0;
    __syncthreads();
    LeafCache lc;
    lc.hist = s_hist;
    if (P.n_big > 0) pivot_block_phase<PV>(P, psmem, sh, ss, lc);
    __syncthreads();
    if (P.n_work > P.n_big) {
        PNest* ws = reinterpret_cast<PNest*>(psmem) + (threadIdx.x >> 5);
        pivot_warp_phase<PV>(P, *ws, lc);
    }
    __syncthreads();
    if (P.gq_cap) pivot_global_phase<PV>(P, psmem, sh, ss, lc);
    if ((threadIdx.x & 31) == 0) {
        lc.flush(P);
        if (lc.nodes) atomicAdd(&P.ctl->words, lc.nodes);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < LH * LQ; i += PB)
        if (s_hist[i]) atomicAdd(&P.leaves[(size_t)(i / LQ) * P.hq + (i % LQ)], s_hist[i]);
}

typedef unsigned __int128 u128;
static constexpr u128 SAT128 = ~(u128)0;

__device__ __forceinline__ u128 sat_add128(u128 a, u128 b) {
    const u128 s = a + b;
    return (s < a || a == SAT128 || b == SAT128) ? SAT128 : s;
}

// Pascal's triangle C(a, b) for a, b < B: t128 exact below 2^128 (SAT128 =
// not representable), t64 the same saturated at 2^64 - 1 (SAT).
__global__ void k_binom(unsigned long long* t64, u128* t128, uint32_t B) {
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) t128[b] = b == 0 ? (u128)1 : (u128)0;
    __syncthreads();
    for (uint32_t a = 1; a < B; ++a) {
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
            const u128 x = b ? t128[(size_t)(a - 1) * B + b - 1] : (u128)0;
            const u128 y = t128[(size_t)(a - 1) * B + b];
            t128[(size_t)a * B + b] = b == 0 ? (u128)1 : sat_add128(x, y);
        }
        __syncthreads();
    }
    for (size_t i = threadIdx.x; i < (size_t)B * B; i += blockDim.x) {
        const u128 c = t128[i];
        t64[i] = (c >> 64) ? SAT : (unsigned long long)c;
    }
}

// counts[j] = sum over (h, q) of leaves[h][q] * C(q, j - h) in 128-bit
// arithmetic (counts_lo / counts_hi); ovf128[j] = 1 when the exact value
// exceeds 2^128 - 1.  omega = max h + q.
__global__ void k_pivot_reduce(const unsigned long long* leaves, uint32_t hq, const u128* binom128, uint32_t B,
                               uint32_t cap, uint32_t kfix, unsigned long long n, unsigned long long m,
                               unsigned long long* counts_lo, unsigned long long* counts_hi, unsigned char* ovf128,
                               unsigned int* omega) {
    for (uint32_t j = threadIdx.x + blockIdx.x * blockDim.x; j < cap; j += gridDim.x * blockDim.x) {
        u128 s = 0;
        bool o = false;
        if (j == 0) s = 1;
        else if (j == 1) s = n;
        else if (j == 2) s = m;
        else if (kfix == 0 || j == kfix) {
            for (uint32_t h = 1; h <= j && h < hq; ++h) {
                for (uint32_t q = j - h; q < hq; ++q) {
                    const unsigned long long L = leaves[(size_t)h * hq + q];
                    if (!L) continue;
                    const u128 c = (q < B && j - h < B) ? binom128[(size_t)q * B + (j - h)] : SAT128;
                    if (c == SAT128) { o = true; continue; }
                    // L * c with c = (chi, clo): L * clo is exact in 128 bits; L * chi must fit in 64
                    const unsigned long long clo = (unsigned long long)c, chi = (unsigned long long)(c >> 64);
                    const u128 p1 = (u128)L * clo;
                    if (chi && __umul64hi(L, chi)) { o = true; continue; }
                    const unsigned long long p2 = L * chi;
                    const unsigned long long top = (unsigned long long)(p1 >> 64) + p2;
                    if (top < p2) { o = true; continue; }
                    const u128 prod = ((u128)top << 64) | (unsigned long long)p1;
                    const u128 t = s + prod;
                    if (t < s) o = true;
                    s = t;
                }
            }
        }
        counts_lo[j] = (unsigned long long)s;
        counts_hi[j] = (unsigned long long)(s >> 64);
        ovf128[j] = o ? 1 : 0;
    }
    if (blockIdx.x == 0) {
        unsigned int w = 0;
        for (size_t x = threadIdx.x; x < (size_t)hq * hq; x += blockDim.x)
            if (leaves[x]) w = max(w, (unsigned)(x / hq + x % hq));
        for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
        if ((threadIdx.x & 31) == 0) atomicMax(omega, w);
    }
}

__global__ void k_pivot_pv_small(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t k,
                                 unsigned long long* pv) {
    // k = 1: every vertex is in one 1-clique; k = 2: its degree (out + in)
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (k == 1) pv[v] = 1;
        else atomicAdd(&pv[v], (unsigned long long)(rp[v + 1] - rp[v]));
    }
    if (k == 2)
        for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
            for (uint32_t e = rp[v]; e < rp[v + 1]; ++e) atomicAdd(&pv[col[e]], 1ull);
}

__global__ void k_map_pv(const unsigned long long* pv, const uint32_t* new_of_old, uint32_t n,
                         unsigned long long* out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = pv[new_of_old[v]];
}

__global__ void k_pivot_set_deadline(Ctl* ctl, unsigned long long budget_ns) {
    ctl->deadline = budget_ns ? globaltimer_ns() + budget_ns : 0ull;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static uint64_t roots_at_least(const kc_graph* g, uint64_t dmin) {
    uint64_t c = 0;
    for (uint64_t d = dmin; d < g->outdeg_hist.size(); ++d) c += g->outdeg_hist[d];
    return c;
}

static constexpr size_t PSMEM_LIMIT = 200 * 1024;  // dynamic; static shared memory comes on top

static kc_status pivot_run(kc_graph* g, uint32_t kfix, uint32_t cap, uint32_t pvk, uint64_t* per_vertex_dev,
                           unsigned long long* counts_dev, unsigned char* ovf_dev, unsigned int* omega_dev,
                           unsigned int* flags_dev, cudaStream_t s) {
    const int sms = g->sm_count;
    const uint32_t n = g->n;
    const uint32_t dcap = std::max<uint32_t>(g->d_max, 1);
    const uint32_t wcap = (dcap + 31) / 32;
    if (dcap >= 0xFFFFu) return set_error(KC_E_UNSUPPORTED, "pivoting supports out-degrees below 65535");
    const uint32_t hq = dcap + 3;        // h, q <= clique number <= d_max + 1
    const uint32_t B = std::max<uint32_t>(dcap + 3, cap + 2);
    const uint32_t dmin = kfix ? std::max<uint32_t>(2, kfix - 1) : 2;
    const uint64_t n_work = roots_at_least(g, dmin);
    const uint64_t n_big = roots_at_least(g, std::max<uint32_t>(PSMALL + 1, dmin));
    // memory: ctl, leaves, binomials, per-root task counters, per-vertex accumulators
    KC_CHECK(dev_alloc(g->ctl, ctl_bytes()));
    Ctl* ctl = (Ctl*)g->ctl.ptr;
    const size_t leaves_b = (size_t)hq * hq * 8, binom_b = (size_t)B * B * 8;
    const size_t tasks_b = ((size_t)n_big + 16) * 4, pv_b = pvk ? ((size_t)n + 16) * 8 : 0;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    KC_CHECK(dev_alloc(g->pv, al(leaves_b) + al(binom_b) + al(2 * binom_b) + al(tasks_b) + al(pv_b)));
    char* p = (char*)g->pv.ptr;
    unsigned long long* leaves = (unsigned long long*)p; p += al(leaves_b);
    unsigned long long* binom_t = (unsigned long long*)p; p += al(binom_b);
    u128* binom128 = (u128*)p; p += al(2 * binom_b);
    uint32_t* tasks = (uint32_t*)p; p += al(tasks_b);
    unsigned long long* pv = pvk ? (unsigned long long*)p : nullptr;
    KC_CUDA(cudaMemsetAsync(ctl, 0, ctl_bytes(), s));
    KC_CUDA(cudaMemsetAsync(leaves, 0, leaves_b, s));
    KC_CUDA(cudaMemsetAsync(tasks, 0, tasks_b, s));
    if (pv) KC_CUDA(cudaMemsetAsync(pv, 0, pv_b, s));
    k_binom<<<1, 1024, 0, s>>>(binom_t, binom128, B);
    note_launch();
    KC_CUDA(cudaGetLastError());
    unsigned long long budget = g->time_limit_s > 0 ? (unsigned long long)(g->time_limit_s * 1e9) : 0ull;
    k_pivot_set_deadline<<<1, 1, 0, s>>>(ctl, budget);
    note_launch();
    KC_CUDA(cudaGetLastError());
    // geometry: candidates, adjacency (if it fits), per-warp start sets,
    // frame queue, paths, one-word-row scratch, then as many wide stack levels
    // per warp as fit in shared memory (the rest in global memory)
    const size_t D0 = (dcap + 31) & ~31u;
    const size_t adj_w = (size_t)dcap * wcap;
    const size_t stride = 2 * (size_t)wcap + HDR;
    const size_t tail_w = wcap + 32 + (size_t)PW * wcap + (size_t)PQCAP * pq_stride(wcap) + (size_t)PW * PPATH +
                          (size_t)PW * (sizeof(PNest) / 4);
    const size_t limit_w = PSMEM_LIMIT / 4;
    int adj_in_smem = 1;
    size_t fixed_w = D0 + adj_w + tail_w;
    if (fixed_w + (size_t)PW * 8 * stride > limit_w) {
        adj_in_smem = 0;
        fixed_w = D0 + tail_w;
    }
    const uint32_t lvl_cap = dcap + 3;
    // nodes with more than 32 candidates are rare below the root (smaller ones
    // move to one-word rows), so a few shared-memory levels per warp suffice;
    // deeper wide levels live in global memory
    uint32_t lvl_smem = (uint32_t)std::min<size_t>(
        std::min<size_t>(lvl_cap, 16), fixed_w < limit_w ? (limit_w - fixed_w) / (PW * stride) : 0);
    const size_t smem_w = fixed_w + (size_t)PW * lvl_smem * stride;
    size_t smem = std::max(smem_w * 4, sizeof(PNest) * PW);
    const bool pvon = pv != nullptr && pvk >= 3;
    void (*kern)(const PivotParams) = pvon ? k_count_pivot<true> : k_count_pivot<false>;
    KC_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int bps = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, PB, smem));
    if (bps < 1) return set_error(KC_E_UNSUPPORTED, "pivot kernel cannot be resident (smem %zu)", smem);
    const int blocks = bps * sms;
    const size_t gstack_words = (((size_t)(lvl_cap - lvl_smem) + 1) * stride + 63) & ~(size_t)63;
    const size_t gadj_words = adj_in_smem ? 0 : ((adj_w + 63) & ~(size_t)63);
    const uint32_t gq_cap = n_big ? 256u : 0u;
    const uint32_t gq_stride = (pq_stride(wcap) + 3) & ~3u;
    const size_t gq_words = (size_t)gq_cap * gq_stride + gq_cap;
    KC_CHECK(dev_alloc(g->scratch,
                       ((size_t)blocks * PW * gstack_words + (size_t)blocks * gadj_words + gq_words + 64) * 4));
    PivotParams P;
    memset(&P, 0, sizeof(P));
    P.rp = (const uint32_t*)g->row_ptr.ptr;
    P.col = (const uint32_t*)g->col.ptr;
    P.roots = (const uint32_t*)g->roots.ptr;
    P.n_big = (uint32_t)n_big;
    P.n_work = (uint32_t)n_work;
    P.n = n;
    P.task_next = tasks;
    P.kfix = kfix;
    P.pvk = pvon ? pvk : 0;
    P.pv = pv;
    P.binom = binom_t;
    P.bstride = B;
    P.leaves = leaves;
    P.hq = hq;
    P.dcap = dcap;
    P.wcap = wcap;
    P.lvl_cap = lvl_cap;
    P.lvl_smem = lvl_smem;
    P.adj_in_smem = adj_in_smem;
    P.gstack = (uint32_t*)g->scratch.ptr;
    P.gstack_words = gstack_words;
    P.gadj = (uint32_t*)g->scratch.ptr + (size_t)blocks * PW * gstack_words;
    P.gadj_words = gadj_words;
    P.gq = P.gadj + (size_t)blocks * gadj_words;
    P.gq_state = P.gq + (size_t)gq_cap * gq_stride;
    P.gq_cap = gq_cap;
    P.gq_stride = gq_stride;
    P.ctl = ctl;
    if (gq_cap) {
        KC_CUDA(cudaMemsetAsync(P.gq_state, 0, (size_t)gq_cap * 4, s));
        const unsigned active = (unsigned)blocks;
        PWorkCtl* wc = reinterpret_cast<PWorkCtl*>(ctl + 1);
        KC_CUDA(cudaMemcpyAsync(&wc->g_active, &active, 4, cudaMemcpyHostToDevice, s));
    }
    if (n_work > 0) {
        kern<<<blocks, PB, smem, s>>>(P);
        note_launch();
        KC_CUDA(cudaGetLastError());
    }
    if (pv && pvk < 3) {
        k_pivot_pv_small<<<std::max(1, sms * 4), 256, 0, s>>>(P.rp, P.col, n, pvk, pv);
        note_launch();
        KC_CUDA(cudaGetLastError());
    }
    KC_CUDA(cudaMemsetAsync(omega_dev, 0, 4, s));
    k_pivot_reduce<<<std::max<uint32_t>(1, (cap + 255) / 256), 256, 0, s>>>(
        leaves, hq, binom128, B, cap, kfix, n, g->m, counts_dev, counts_dev + cap, ovf_dev, omega_dev);
    note_launch();
    KC_CUDA(cudaGetLastError());
    if (per_vertex_dev && pv) {
        k_map_pv<<<std::max(1, sms * 4), 256, 0, s>>>(pv, (const uint32_t*)g->new_of_old.ptr, n,
                                                       (unsigned long long*)per_vertex_dev);
        note_launch();
        KC_CUDA(cudaGetLastError());
    }
    KC_CUDA(cudaMemcpyAsync(flags_dev, &ctl->flags, 4, cudaMemcpyDeviceToDevice, s));
    return KC_OK;
}

__global__ void k_pack_pivot_result(const unsigned long long* counts, uint32_t cap, const unsigned char* ovf128,
                                    const unsigned* flags, const Ctl* ctl, uint32_t k, kc_result* out) {
    kc_result r;
    r.total = counts[k];
    r.total_hi = counts[cap + k];
    r.flags = *flags;
    if (r.total_hi || ovf128[k]) r.flags |= KC_FLAG_TOTAL_OVERFLOW;
    if (ovf128[k]) r.flags |= KC_FLAG_TOTAL_OVERFLOW128;
    r.status = (*flags & KC_FLAG_TIMEOUT) ? KC_E_TIMEOUT : ((*flags & KC_FLAG_INTERNAL) ? KC_E_INTERNAL : KC_OK);
    r.words = ctl->words;
    *out = r;
}

// Output area of a pivoting run: counts lo[cap], hi[cap] (u64 each),
// ovf128[cap] u8, omega, flags.
static kc_status pivot_out(kc_graph* g, uint32_t cap, unsigned long long*& counts, unsigned char*& ovf,
                           unsigned int*& omega, unsigned int*& flags) {
    const size_t cb = ((size_t)cap * 16 + 255) & ~(size_t)255, ob = ((size_t)cap + 255) & ~(size_t)255;
    KC_CHECK(dev_alloc(g->pivot_out, cb + ob + 256));
    char* p = (char*)g->pivot_out.ptr;
    counts = (unsigned long long*)p;
    ovf = (unsigned char*)(p + cb);
    omega = (unsigned int*)(p + cb + ob);
    flags = omega + 1;
    return KC_OK;
}

kc_status count_pivot_async(kc_graph* g, uint32_t k, kc_result* result_dev, uint64_t* per_vertex_dev,
                            cudaStream_t s) {
    unsigned long long* counts;
    unsigned char* ovf;
    unsigned int *omega, *flags;
    KC_CHECK(pivot_out(g, k + 1, counts, ovf, omega, flags));
    KC_CHECK(pivot_run(g, k, k + 1, per_vertex_dev ? k : 0, per_vertex_dev, counts, ovf, omega, flags, s));
    k_pack_pivot_result<<<1, 1, 0, s>>>(counts, k + 1, ovf, flags, (const Ctl*)g->ctl.ptr, k, result_dev);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status count_all_run(kc_graph* g, uint32_t cap, uint32_t pvk, uint64_t* per_vertex_dev, uint64_t* counts_lo_host,
                        uint64_t* counts_hi_host, uint8_t* ovf128_host, uint32_t* omega_host, uint32_t* flags_host,
                        cudaStream_t s) {
    unsigned long long* counts;
    unsigned char* ovf;
    unsigned int *omega, *flags;
    KC_CHECK(pivot_out(g, cap, counts, ovf, omega, flags));
    KC_CHECK(pivot_run(g, 0, cap, pvk, per_vertex_dev, counts, ovf, omega, flags, s));
    KC_CUDA(cudaMemcpyAsync(counts_lo_host, counts, (size_t)cap * 8, cudaMemcpyDeviceToHost, s));
    if (counts_hi_host) KC_CUDA(cudaMemcpyAsync(counts_hi_host, counts + cap, (size_t)cap * 8, cudaMemcpyDeviceToHost, s));
    if (ovf128_host) KC_CUDA(cudaMemcpyAsync(ovf128_host, ovf, cap, cudaMemcpyDeviceToHost, s));
    unsigned int of[2];
    KC_CUDA(cudaMemcpyAsync(of, omega, 8, cudaMemcpyDeviceToHost, s));
    unsigned long long work = 0;
    KC_CUDA(cudaMemcpyAsync(&work, &((const Ctl*)g->ctl.ptr)->words, 8, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    g->last_work = work;
    uint32_t om = of[0];
    if (g->m > 0 && om < 2) om = 2;
    if (g->n > 0 && om < 1) om = 1;
    if (omega_host) *omega_host = om;
    if (flags_host) *flags_host = of[1];
    return KC_OK;
}

}  // namespace kc
