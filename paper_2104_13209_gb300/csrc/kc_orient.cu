// Graph orientation (Section 3.1): validate the input CSR, compute the
// orientation key (degree, or the peel round of a level-synchronous k-core
// decomposition), turn it into a vertex order, keep only the edges that go
// forward in that order, rebuild the row pointers by histogram + exclusive
// scan, and sort every DAG row.
//
// The DAG is stored in the library numbering: vertex r is the r-th vertex of
// the order, so every edge goes from a smaller to a larger id.  The induced
// sub-graph of any candidate set listed in ascending id is then strictly
// upper-triangular, which the counting kernels rely on.

#include <algorithm>
#include <mutex>

#include "kc_common.cuh"

namespace kc {

static constexpr uint32_t UNSET = 0xFFFFFFFFu;

// Flags of the validation pass.
enum : unsigned {
    VF_ROWPTR = 1u,     // row_ptr not monotone, row_ptr[0] != 0 or row_ptr[n] != nnz
    VF_RANGE = 2u,      // an id >= n
    VF_SELFLOOP = 4u,   // u in N(u)
    VF_ORDER = 8u,      // a row not strictly ascending (includes duplicates)
    VF_ASYM = 16u,      // (u, v) present but (v, u) absent
};

__device__ __forceinline__ uint32_t row_of_entry(const uint32_t* rp, uint32_t n, uint32_t e) {
    // largest u with rp[u] <= e (rp monotone, e < rp[n])
    uint32_t lo = 0, hi = n;  // answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (rp[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains_sorted(const uint32_t* a, uint32_t len, uint32_t x) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint32_t y = a[mid];
        if (y == x) return true;
        if (y < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

__global__ void k_validate_rowptr(const uint32_t* __restrict__ rp, uint32_t n, uint64_t nnz, unsigned* flags) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        if (rp[u] > rp[u + 1]) atomicOr(flags, VF_ROWPTR);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        if (rp[0] != 0 || (uint64_t)rp[n] != nnz) atomicOr(flags, VF_ROWPTR);
}

// Each thread checks 8 consecutive entries.
__global__ void k_validate_entries(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci, uint32_t n,
                                   uint32_t nnz, unsigned* flags) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t e0 = t * 8;
    if (e0 >= nnz) return;
    uint32_t e = (uint32_t)e0;
    uint32_t end = (uint32_t)(e0 + 8 < (uint64_t)nnz ? e0 + 8 : (uint64_t)nnz);
    uint32_t u = row_of_entry(rp, n, e);
    unsigned f = 0;
    for (; e < end; ++e) {
        while (rp[u + 1] <= e) ++u;
        uint32_t v = ci[e];
        if (v >= n) { f |= VF_RANGE; continue; }
        if (v == u) f |= VF_SELFLOOP;
        if (e > rp[u] && ci[e - 1] >= v) f |= VF_ORDER;
        if (!contains_sorted(ci + rp[v], rp[v + 1] - rp[v], u)) f |= VF_ASYM;
    }
    if (f) atomicOr(flags, f);
}

__global__ void k_degree_key(const uint32_t* __restrict__ rp, uint32_t n, uint32_t* __restrict__ key,
                             int* __restrict__ deg, uint32_t* __restrict__ round_of, unsigned* maxkey) {
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t mx = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t d = rp[v + 1] - rp[v];
        if (key) key[v] = d;
        if (deg) deg[v] = (int)d;
        if (round_of) round_of[v] = UNSET;
        mx = max(mx, d);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxkey, mx);
}

// ---------------------------------------------------------------------------
// Level-synchronous k-core peeling in one thread-block cluster.
//
// At level L every remaining vertex of degree <= L is removed in sub-rounds:
// a scan of the remaining vertices takes those of degree <= L (the first
// frontier), then each sub-round removes a frontier, decrements the degrees
// of all its neighbours, and a neighbour whose degree falls from L + 1 to L
// joins the next frontier.  When a sub-round pushes nothing, L grows by one
// (or jumps to the smallest remaining degree when a scan takes nothing).
// A vertex's core number is the level at which it leaves; its first
// orientation key is its sub-round (round_of).  A vertex removed at level L
// had at most L neighbours left at the start of its sub-round, so the DAG
// that orients edges by (sub-round, ...) has out-degree <= degeneracy.
//
// The peel is a chain of short phases (R-MAT scale 20: about 170 levels and
// 630 sub-rounds), so the time between phases dominates, not the 31 M
// neighbour decrements.  One cluster of up to 16 blocks runs it: the phases
// are separated by hardware cluster barriers, and the control words live in
// the shared memory of the cluster's first block (distributed shared
// memory).  Frontiers are lists of items of at most PEEL_CH adjacency
// entries, so a hub's neighbours spread over many lanes and every phase
// needs one barrier.
//
// Control words rotate over three slots: phase p reads slot p % 3 (written
// during phase p - 1), adds to slot (p + 1) % 3, and clears slot
// (p + 2) % 3, whose last reader finished before the barrier that opened
// phase p.  Every thread takes the same decision from the slot it reads, so
// the loop stays uniform over the cluster.
//
// Degrees are decremented unconditionally (a removed vertex can never again
// cross from L + 1 to L), so they say nothing about removed vertices; the
// second orientation key, the remaining degree at removal, is computed after
// the peel by k_removal_key: #{w in N(v) : round_of[w] >= round_of[v]}.
// ---------------------------------------------------------------------------
static constexpr uint32_t PEEL_CH = 16;        // adjacency entries per frontier item
static constexpr int SCAN_PER_LANE = 8;        // remaining-list entries per lane and round of a scan
static constexpr int PROC_STEP = 8;            // adjacency entries a lane decrements at once
static constexpr int PEEL_THREADS = 1024;

struct PeelSlot {
    unsigned items;   // frontier items pushed during the phase
    unsigned taken;   // vertices removed during the phase
    unsigned kept;    // remaining-list entries written (scan phases)
    unsigned minrem;  // smallest degree among the kept vertices (scan phases)
    unsigned err;     // KC_FLAG_INTERNAL raised during the phase
};

// Result of the peel, read by the host.
struct PeelOut {
    unsigned flags;
    unsigned max_level;   // the degeneracy
    unsigned rounds;      // number of sub-rounds (largest round_of + 1)
    unsigned phases;
};

// Warp-aggregated add to a counter; returns this lane's offset (all lanes call).
__device__ __forceinline__ unsigned warp_reserve(unsigned cnt, unsigned* counter) {
    const int lane = threadIdx.x & 31;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - cnt;
}

// Lanes with pred[u] remove vertex v[u] now (sub-round `round`, level
// `level`): mark it, then append its adjacency as frontier items to F
// (capacity fcap, item count in sl->items), N candidates per lane at once:
// the rows' bounds are loaded together, and the warp reserves the items of
// all its takes with one atomic (a phase's reservations are the peel's
// only contended atomics).  All lanes call.
template <int N>
__device__ __forceinline__ void peel_take_many(const bool (&pred)[N], const uint32_t (&v)[N], uint32_t round,
                                               uint32_t level, const uint32_t* __restrict__ rp, uint32_t* round_of,
                                               uint32_t* core, uint2* F, uint32_t fcap, PeelSlot* sl) {
    uint32_t b[N], len[N];
    uint32_t tot = 0, nt = 0;
#pragma unroll
    for (int u = 0; u < N; ++u) {
        b[u] = 0;
        len[u] = 0;
        if (pred[u]) {
            __stcg(&round_of[v[u]], round);
            __stcg(&core[v[u]], level);
            b[u] = __ldg(rp + v[u]);
            len[u] = __ldg(rp + v[u] + 1);
        }
    }
#pragma unroll
    for (int u = 0; u < N; ++u)
        if (pred[u]) {
            len[u] -= b[u];
            tot += (len[u] + PEEL_CH - 1) / PEEL_CH;
            ++nt;
        }
    const unsigned any = __ballot_sync(0xffffffffu, nt > 0);
    if (any == 0) return;
    const int lane = threadIdx.x & 31;
    const unsigned ntw = __reduce_add_sync(0xffffffffu, nt);
    if (lane == __ffs(any) - 1) atomicAdd(&sl->taken, ntw);
    uint32_t off = warp_reserve(tot, &sl->items);
#pragma unroll
    for (int u = 0; u < N; ++u) {
        const uint32_t c = (len[u] + PEEL_CH - 1) / PEEL_CH;
        unsigned m = __ballot_sync(0xffffffffu, c > 0);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t sb = __shfl_sync(0xffffffffu, b[u], src), sl2 = __shfl_sync(0xffffffffu, len[u], src);
            const uint32_t sc = __shfl_sync(0xffffffffu, c, src), so = __shfl_sync(0xffffffffu, off, src);
            for (uint32_t x = lane; x < sc; x += 32) {
                const uint32_t pos = so + x;
                if (pos < fcap) __stcg(&F[pos], make_uint2(sb + x * PEEL_CH, min(PEEL_CH, sl2 - x * PEEL_CH)));
                else atomicOr(&sl->err, (unsigned)KC_FLAG_INTERNAL);
            }
        }
        off += c;
    }
}

// Loop state of the peel, the same in every thread of the cluster.
struct PeelState {
    uint32_t level, round, p, max_level;
    uint32_t nf;    // items of the frontier the next process phase reads
    uint32_t rn;    // entries of the remaining list the next scan reads
    uint32_t fail;  // KC_FLAG_* when the loop stopped on an inconsistency
    int fb;         // frontier buffer the next phase pushes into
    int pf;         // frontier buffer the next process phase reads
    int rl;         // remaining list the next scan reads
    int all;        // the next scan reads every vertex (the first one)
    int scan;       // kind of the next phase
    int done;
};

// Phases at most this large run in the cluster's first block alone, with
// block barriers between them, while the other blocks wait at one cluster
// barrier: most of the peel's phases are tiny frontiers of the long tail.
static constexpr uint32_t SOLO_SCAN = 8192;   // remaining-list entries of a scan
static constexpr uint32_t SOLO_ITEMS = 1024;  // frontier items of a process phase

__device__ __forceinline__ bool peel_small(const PeelState& S) {
    return S.scan ? S.rn <= SOLO_SCAN : S.nf <= SOLO_ITEMS;
}

// One phase of the peel by the threads given (gwarp of nwarps warps):
// adds to the control slot wr.
__device__ __forceinline__ void peel_phase(const PeelState& S, uint32_t gwarp, uint32_t nwarps,
                                           const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci,
                                           uint32_t n, int* deg, uint32_t* round_of, uint32_t* core, uint2* F0,
                                           uint2* F1, uint32_t fcap, uint32_t* R0, uint32_t* R1, PeelSlot* wr) {
    const uint32_t lane = threadIdx.x & 31;
    if (S.scan) {
        // take the remaining vertices of degree <= level, keep the others;
        // a lane looks at SCAN_PER_LANE entries per round (their loads in
        // flight together) and the warp reserves the kept ones at once
        uint32_t local_min = UNSET;
        uint32_t* Rw = S.rl ? R0 : R1;
        const uint32_t* Rr = S.rl ? R1 : R0;
        uint2* Fw = S.fb ? F1 : F0;
        const uint32_t span = 32u * SCAN_PER_LANE;
        for (unsigned long long base = (unsigned long long)gwarp * span; base < S.rn;
             base += (unsigned long long)nwarps * span) {
            uint32_t v[SCAN_PER_LANE], r[SCAN_PER_LANE];
            int d[SCAN_PER_LANE];
#pragma unroll
            for (int u = 0; u < SCAN_PER_LANE; ++u) {
                const unsigned long long idx = base + (uint32_t)u * 32u + lane;
                v[u] = idx < S.rn ? (S.all ? (uint32_t)idx : __ldcg(&Rr[idx])) : UNSET;
            }
#pragma unroll
            for (int u = 0; u < SCAN_PER_LANE; ++u) {
                r[u] = v[u] != UNSET ? __ldcg(&round_of[v[u]]) : 0u;
                d[u] = v[u] != UNSET ? __ldcg(&deg[v[u]]) : 0;
            }
            unsigned keepm = 0, nkeep = 0;
            bool take[SCAN_PER_LANE];
#pragma unroll
            for (int u = 0; u < SCAN_PER_LANE; ++u) {
                const bool live = v[u] != UNSET && r[u] == UNSET;
                take[u] = live && d[u] <= (int)S.level;
                if (live && !take[u]) {
                    keepm |= 1u << u;
                    ++nkeep;
                    local_min = min(local_min, (uint32_t)d[u]);
                }
            }
            peel_take_many<SCAN_PER_LANE>(take, v, S.round, S.level, rp, round_of, core, Fw, fcap, wr);
            uint32_t o = warp_reserve(nkeep, &wr->kept);
#pragma unroll
            for (int u = 0; u < SCAN_PER_LANE; ++u)
                if (keepm >> u & 1u) {
                    if (o < n) __stcg(&Rw[o], v[u]);
                    else atomicOr(&wr->err, (unsigned)KC_FLAG_INTERNAL);
                    ++o;
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
        if (lane == 0 && local_min != UNSET) atomicMin(&wr->minrem, local_min);
    } else {
        // remove frontier pf: decrement every neighbour of its items; a
        // neighbour that falls to the level joins frontier fb
        const uint2* Fr = S.pf ? F1 : F0;
        uint2* Fw = S.fb ? F1 : F0;
        for (uint32_t base = gwarp * 32; base < S.nf; base += nwarps * 32) {
            const uint32_t i = base + lane;
            uint2 it = make_uint2(0u, 0u);
            if (i < S.nf) it = __ldcg(&Fr[i]);
            for (uint32_t t0 = 0; t0 < PEEL_CH; t0 += PROC_STEP) {
                if (__ballot_sync(0xffffffffu, it.y > t0) == 0) break;
                uint32_t w[PROC_STEP];
                int old[PROC_STEP];
                bool take[PROC_STEP];
#pragma unroll
                for (int u = 0; u < PROC_STEP; ++u) w[u] = (t0 + u < it.y) ? __ldg(ci + it.x + t0 + u) : UNSET;
#pragma unroll
                for (int u = 0; u < PROC_STEP; ++u) old[u] = (w[u] < n) ? atomicSub(&deg[w[u]], 1) : 0;
#pragma unroll
                for (int u = 0; u < PROC_STEP; ++u) take[u] = w[u] < n && old[u] == (int)S.level + 1;
                peel_take_many<PROC_STEP>(take, w, S.round + 1, S.level, rp, round_of, core, Fw, fcap, wr);
            }
        }
    }
}

// The loop's decisions after a phase, from the slot c it wrote.
__device__ __forceinline__ void peel_advance(PeelState& S, const PeelSlot& c, uint32_t n, uint32_t fcap,
                                             uint32_t phase_cap) {
    if (c.err) {
        S.fail = c.err;
        S.done = 1;
        return;
    }
    if (S.p > phase_cap) {
        S.fail = KC_FLAG_INTERNAL;
        S.done = 1;
        return;
    }
    if (S.scan) {
        if (c.taken) S.max_level = S.level;
        S.rl ^= 1;
        S.rn = min(c.kept, n);
        S.all = 0;
        S.nf = min(c.items, fcap);
        if (S.nf == 0) {
            if (S.rn == 0) {  // every vertex is removed
                S.done = 1;
                return;
            }
            // nothing (with edges) left at this level: jump to the smallest remaining degree
            if (c.minrem == UNSET || c.minrem <= S.level) {
                S.fail = KC_FLAG_INTERNAL;
                S.done = 1;
                return;
            }
            S.level = c.minrem;
        } else {
            S.pf = S.fb;
            S.fb ^= 1;
            S.scan = 0;
        }
    } else {
        ++S.round;
        S.nf = min(c.items, fcap);
        if (S.nf == 0) {
            ++S.level;
            S.scan = 1;
        } else {
            S.pf = S.fb;
            S.fb ^= 1;
        }
    }
}

// Global control words of the peel (device memory, set up by the kernel).
struct PeelCtl {
    PeelSlot slot[3];  // control slots of the grid-wide phases
    PeelState pub;     // block 0's loop state after it ran phases alone
    unsigned bar;      // barrier arrivals since the launch
    unsigned fail;     // KC_FLAG_INTERNAL: a barrier wait gave up
};

// A barrier wait gives up after this long (%globaltimer); the first one,
// which also waits for every block of the launch to start (blocks of other
// kernels may hold SMs until they finish), after START.
static constexpr unsigned long long PEEL_BARRIER_NS = 2000000000ull;
static constexpr unsigned long long PEEL_START_NS = 60000000000ull;

// Grid-wide barrier of the peel: arrivals only count up, and a block waits
// until the count reaches its target (gridDim.x more per barrier), so no
// reset is needed.  Returns false (and records KC_FLAG_INTERNAL) when the
// wait gives up; the caller then leaves its loop, and the other blocks' next
// waits give up too, so the launch always ends.
__device__ __forceinline__ bool peel_barrier(PeelCtl* pc, unsigned target, unsigned long long limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        __threadfence();
        atomicAdd(&pc->bar, 1u);
        if (*(volatile unsigned*)&pc->bar < target) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned spins = 0;
            while (*(volatile unsigned*)&pc->bar < target) {
                if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) {
                    atomicOr(&pc->fail, (unsigned)KC_FLAG_INTERNAL);
                    good = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ PeelSlot load_slot(const PeelSlot* p) {
    const volatile unsigned* w = reinterpret_cast<const volatile unsigned*>(p);
    return PeelSlot{w[0], w[1], w[2], w[3], w[4]};
}

// The peel over every SM: one block of PEEL_THREADS per SM, all resident
// (cooperative launch).  Large phases run on the whole grid with grid-wide
// barriers between them; runs of small phases run in block 0 alone, with
// block barriers, while the other blocks wait at one grid barrier.
__global__ void __launch_bounds__(PEEL_THREADS, 1)
k_peel_grid(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci, uint32_t n, int* deg,
            uint32_t* round_of, uint32_t* core, uint2* F0, uint2* F1, uint32_t fcap, uint32_t* R0, uint32_t* R1,
            PeelCtl* pc, PeelOut* out) {
    __shared__ PeelSlot slots[3];  // block 0's phases alone
    __shared__ PeelSlot seen;      // the slot read after a grid barrier
    __shared__ PeelState got;
    const PeelSlot clean{0u, 0u, 0u, UNSET, 0u};
    const unsigned nblk = gridDim.x;
    const uint32_t gwarp = blockIdx.x * (PEEL_THREADS / 32) + (threadIdx.x >> 5);
    const uint32_t nwarps = nblk * (PEEL_THREADS / 32);
    const uint32_t phase_cap = 4u * n + 64u;
    if (blockIdx.x == 0 && threadIdx.x < 3) pc->slot[threadIdx.x] = clean;
    unsigned target = nblk;
    bool ok = peel_barrier(pc, target, PEEL_START_NS);
    PeelState S;
    S.level = 0;
    S.round = 0;
    S.p = 0;
    S.max_level = 0;
    S.nf = 0;
    S.rn = n;
    S.fail = 0;
    S.fb = 0;
    S.pf = 1;
    S.rl = 0;
    S.all = 1;
    S.scan = 1;
    S.done = 0;
    while (ok) {
        if (nblk > 1 && peel_small(S)) {
            if (blockIdx.x == 0) {
                if (threadIdx.x < 3) slots[threadIdx.x] = clean;
                __syncthreads();
                for (;;) {
                    PeelSlot* wr = slots + (S.p + 1) % 3;
                    if (threadIdx.x == 0) slots[(S.p + 2) % 3] = clean;
                    peel_phase(S, threadIdx.x >> 5, PEEL_THREADS / 32, rp, ci, n, deg, round_of, core, F0, F1, fcap,
                               R0, R1, wr);
                    __syncthreads();
                    ++S.p;
                    const PeelSlot c = *wr;
                    __syncthreads();  // every thread read the slot before the next phase clears slots
                    peel_advance(S, c, n, fcap, phase_cap);
                    if (S.done || !peel_small(S)) break;
                }
                // the grid-wide phases that follow start from clean slots
                if (threadIdx.x < 3) pc->slot[threadIdx.x] = clean;
                if (threadIdx.x == 0) pc->pub = S;
            }
            target += nblk;
            ok = peel_barrier(pc, target, PEEL_BARRIER_NS);
            if (!ok) break;
            if (blockIdx.x != 0) {
                if (threadIdx.x == 0) {
                    const volatile PeelState* vp = &pc->pub;
                    got.level = vp->level;
                    got.round = vp->round;
                    got.p = vp->p;
                    got.max_level = vp->max_level;
                    got.nf = vp->nf;
                    got.rn = vp->rn;
                    got.fail = vp->fail;
                    got.fb = vp->fb;
                    got.pf = vp->pf;
                    got.rl = vp->rl;
                    got.all = vp->all;
                    got.scan = vp->scan;
                    got.done = vp->done;
                }
                __syncthreads();
                S = got;
            }
            if (S.done) break;
            continue;
        }
        PeelSlot* wr = pc->slot + (S.p + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) pc->slot[(S.p + 2) % 3] = clean;
        peel_phase(S, gwarp, nwarps, rp, ci, n, deg, round_of, core, F0, F1, fcap, R0, R1, wr);
        target += nblk;
        ok = peel_barrier(pc, target, PEEL_BARRIER_NS);
        if (!ok) break;
        ++S.p;
        if (threadIdx.x == 0) seen = load_slot(wr);
        __syncthreads();
        const PeelSlot c = seen;
        peel_advance(S, c, n, fcap, phase_cap);
        if (S.done) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->flags = S.fail | (ok ? 0u : (unsigned)KC_FLAG_INTERNAL) | *(volatile unsigned*)&pc->fail;
        out->max_level = S.max_level;
        out->rounds = S.round + 1;
        out->phases = S.p;
    }
}

// Second orientation key: the remaining degree of v when it was removed,
// #{w in N(v) : round_of[w] >= round_of[v]} (one warp per vertex).
__global__ void k_removal_key(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci, uint32_t n,
                              const uint32_t* __restrict__ round_of, uint32_t* __restrict__ key) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t v = gw; v < n; v += nw) {
        const uint32_t b = rp[v], e = rp[v + 1], r = round_of[v];
        uint32_t c = 0;
        for (uint32_t j = b + lane; j < e; j += 32) c += round_of[ci[j]] >= r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) key[v] = c;
    }
}

// ---------------------------------------------------------------------------
// Relabel + filter
// ---------------------------------------------------------------------------
__global__ void k_invert(const uint32_t* __restrict__ old_of_new, uint32_t n, uint32_t* __restrict__ new_of_old) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) new_of_old[old_of_new[r]] = r;
}

// For 8 consecutive input entries per thread: count the kept (forward) ones
// per library row (mode 0), or write their library ids at the row cursor
// (mode 1).
template <int MODE>
__global__ void k_filter(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci, uint32_t n, uint32_t nnz,
                         const uint32_t* __restrict__ new_of_old, uint32_t* __restrict__ outdeg_or_cursor,
                         uint32_t* __restrict__ out_col) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t e0 = t * 8;
    if (e0 >= nnz) return;
    uint32_t e = (uint32_t)e0;
    uint32_t end = (uint32_t)(e0 + 8 < (uint64_t)nnz ? e0 + 8 : (uint64_t)nnz);
    uint32_t u = row_of_entry(rp, n, e);
    uint32_t ru = new_of_old[u];
    uint32_t cnt = 0;
    for (; e < end; ++e) {
        while (rp[u + 1] <= e) {
            if (MODE == 0 && cnt) atomicAdd(&outdeg_or_cursor[ru], cnt);
            cnt = 0;
            ++u;
            ru = new_of_old[u];
        }
        uint32_t rw = new_of_old[ci[e]];
        if (rw > ru) {
            if (MODE == 0) ++cnt;
            else out_col[atomicAdd(&outdeg_or_cursor[ru], 1u)] = rw;
        }
    }
    if (MODE == 0 && cnt) atomicAdd(&outdeg_or_cursor[ru], cnt);
}

// Out-degree key (for the root order) and out-degree histogram.  Bins below
// OUTDEG_BINS are counted in shared memory first: most vertices have small
// out-degrees, and global atomics on the same few bins would serialise.
static constexpr uint32_t OUTDEG_BINS = 1024;
__global__ void k_outdeg_from_rowptr(const uint32_t* __restrict__ rp, uint32_t n, uint32_t* __restrict__ key,
                                     uint32_t dmax, unsigned* __restrict__ hist) {
    __shared__ unsigned sh[OUTDEG_BINS];
    for (uint32_t i = threadIdx.x; i < OUTDEG_BINS; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        uint32_t d = rp[r + 1] - rp[r];
        key[r] = dmax - d;
        if (d < OUTDEG_BINS) atomicAdd(&sh[d], 1u);
        else atomicAdd(&hist[d], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < OUTDEG_BINS && i <= dmax; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void k_rowlen_max(const uint32_t* __restrict__ rp, uint32_t n, unsigned* __restrict__ mx) {
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t m = 0;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) m = max(m, rp[r + 1] - rp[r]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// Sort every DAG row ascending: bitonic in registers for <= 32 entries, rank
// sort (entries are distinct) through shared memory up to SORT_SMEM, rank sort
// from global memory beyond.  src holds the unsorted rows, dst receives them.
static constexpr int ROWSORT_WARPS = 8;
static constexpr int ROWSORT_SMEM = 1024;

__global__ void __launch_bounds__(ROWSORT_WARPS * 32) k_sort_rows(const uint32_t* __restrict__ rp,
                                                                   const uint32_t* __restrict__ src,
                                                                   uint32_t* __restrict__ dst, uint32_t n) {
    __shared__ uint32_t buf[ROWSORT_WARPS][ROWSORT_SMEM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t gw = blockIdx.x * ROWSORT_WARPS + w, nw = gridDim.x * ROWSORT_WARPS;
    for (uint32_t r = gw; r < n; r += nw) {
        const uint32_t b = rp[r], len = rp[r + 1] - b;
        if (len == 0) continue;
        if (len <= 32) {
            uint32_t x = lane < (int)len ? src[b + lane] : 0xFFFFFFFFu;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
                    bool up = (lane & k) == 0;
                    bool lower = (lane & j) == 0;
                    x = (lower == up) ? min(x, y) : max(x, y);
                }
            }
            if (lane < (int)len) dst[b + lane] = x;
        } else if (len <= ROWSORT_SMEM) {
            for (uint32_t i = lane; i < len; i += 32) buf[w][i] = src[b + i];
            __syncwarp();
            for (uint32_t i = lane; i < len; i += 32) {
                uint32_t x = buf[w][i], rank = 0;
                for (uint32_t j = 0; j < len; ++j) rank += buf[w][j] < x;
                dst[b + rank] = x;
            }
            __syncwarp();
        } else {
            for (uint32_t i = lane; i < len; i += 32) {
                uint32_t x = src[b + i], rank = 0;
                for (uint32_t j = 0; j < len; ++j) rank += src[b + j] < x;
                dst[b + rank] = x;
            }
        }
    }
}


// ---------------------------------------------------------------------------

static unsigned grid_for(uint64_t items, int threads, int sms) {
    uint64_t b = (items + threads - 1) / threads;
    uint64_t cap = (uint64_t)sms * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Blocks of the grid-wide peel: one per SM, provided a block of
// PEEL_THREADS fits an SM and the device runs cooperative launches; looked
// up once per device (0: the device cannot run it).
static kc_status peel_grid_blocks(int sms, int* out) {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || cached[dev] == 0) {
        int coop = 0, per_sm = 0;
        KC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel_grid, PEEL_THREADS, 0));
        const int v = (coop && per_sm >= 1) ? 1 : -1;
        if (dev >= 0 && dev < 64) cached[dev] = v;
        if (v < 0) {
            *out = 0;
            return KC_OK;
        }
    } else if (cached[dev] < 0) {
        *out = 0;
        return KC_OK;
    }
    *out = std::max(1, sms);
    return KC_OK;
}

kc_status build_graph(kc_graph* g, const uint32_t* d_rp, const uint32_t* d_ci, int validate, cudaStream_t s) {
    const uint32_t n = g->n;
    const uint32_t nnz = (uint32_t)(2 * g->m);
    const int sms = g->sm_count;
    cudaEvent_t ev0, ev1;
    KC_CUDA(cudaEventCreate(&ev0));
    KC_CUDA(cudaEventCreate(&ev1));
    KC_CUDA(cudaEventRecord(ev0, s));

    // scratch: small control words + per-vertex arrays
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // frontier items: a vertex of degree d is pushed once, as ceil(d / PEEL_CH) items
    const size_t fcap = (size_t)n + (size_t)nnz / PEEL_CH + 1;
    void* work = nullptr;
    size_t wbytes = al(sizeof(PeelOut)) + al(sizeof(PeelCtl)) + al(64) + 6 * al((size_t)n * 4 + 4) +
                    2 * al(fcap * 8) + al(((size_t)nnz / 2 + 1) * 4);
    kc_status st = scratch_alloc(&work, wbytes, s);
    if (st != KC_OK) return st;
    char* p = (char*)work;
    PeelOut* pout = (PeelOut*)p; p += al(sizeof(PeelOut));
    PeelCtl* pctl = (PeelCtl*)p; p += al(sizeof(PeelCtl));
    unsigned* words = (unsigned*)p; p += al(64);            // [0] validate flags, [1] max key, [2] d_max
    uint32_t* key = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    int* deg = (int*)p; p += al((size_t)n * 4 + 4);
    uint32_t* round_of = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint2* F0 = (uint2*)p; p += al(fcap * 8);                // reused below as u32[n + 1] scratch
    uint2* F1 = (uint2*)p; p += al(fcap * 8);
    uint32_t* heavy = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* R0 = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* R1 = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* colbuf = (uint32_t*)p; p += al(((size_t)nnz / 2 + 1) * 4);

    auto fail = [&](kc_status e) {
        scratch_free(work, s);  // after the kernels queued so far (stream order)
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return e;
    };
#define KC_TRY(call)                                                          \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return fail(cuda_error(e_, #call, __FILE__, __LINE__)); \
    } while (0)
#define KC_TRYS(stcall)                     \
    do {                                    \
        kc_status s2_ = (stcall);           \
        if (s2_ != KC_OK) return fail(s2_); \
    } while (0)

    KC_TRY(cudaMemsetAsync(pout, 0, al(sizeof(PeelOut)) + al(sizeof(PeelCtl)), s));
    KC_TRY(cudaMemsetAsync(words, 0, 64, s));
    unsigned h_words[4] = {0, 0, 0, 0};

    if (validate) {
        k_validate_rowptr<<<grid_for(n, 256, sms), 256, 0, s>>>(d_rp, n, nnz, words);
        note_launch();
        KC_TRY(cudaGetLastError());
        KC_TRY(cudaMemcpyAsync(h_words, words, 4, cudaMemcpyDeviceToHost, s));
        KC_TRY(cudaStreamSynchronize(s));
        if (h_words[0]) return fail(set_error(KC_E_INVALID_GRAPH, "row_ptr is not a valid CSR row pointer array"));
        if (nnz) {
            uint64_t threads = ((uint64_t)nnz + 7) / 8;
            k_validate_entries<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(d_rp, d_ci, n, nnz, words);
            note_launch();
            KC_TRY(cudaGetLastError());
        }
        KC_TRY(cudaMemcpyAsync(h_words, words, 4, cudaMemcpyDeviceToHost, s));
        KC_TRY(cudaStreamSynchronize(s));
        if (h_words[0]) {
            unsigned f = h_words[0];
            return fail(set_error(KC_E_INVALID_GRAPH, "graph is not simple and undirected:%s%s%s%s",
                                  (f & VF_RANGE) ? " vertex id >= n;" : "", (f & VF_SELFLOOP) ? " self-loop;" : "",
                                  (f & VF_ORDER) ? " row not strictly ascending (unsorted or duplicate);" : "",
                                  (f & VF_ASYM) ? " asymmetric adjacency;" : ""));
        }
    }

    // orientation key
    const bool degen = g->orient == KC_ORIENT_DEGENERACY;
    k_degree_key<<<grid_for(n, 256, sms), 256, 0, s>>>(d_rp, n, degen ? nullptr : key, degen ? deg : nullptr,
                                                       degen ? round_of : nullptr, words + 1);
    note_launch();
    KC_TRY(cudaGetLastError());
    uint32_t max_key = 0;
    unsigned maxdeg = 0;  // largest degree (degeneracy order: read with the peel's result)
    if (degen) {
        KC_TRYS(dev_alloc(g->core, (size_t)n * 4 + 4));
        if (n > 0) {
            int blocks = 0;
            KC_TRYS(peel_grid_blocks(sms, &blocks));
            if (blocks == 0) return fail(set_error(KC_E_UNSUPPORTED, "the device cannot run the cooperative k-core peel"));
            const uint32_t fc = (uint32_t)std::min<size_t>(fcap, 0xFFFFFFFFu);
            uint32_t* corep = (uint32_t*)g->core.ptr;
            void* args[] = {(void*)&d_rp, (void*)&d_ci, (void*)&n, (void*)&deg, (void*)&round_of, (void*)&corep,
                            (void*)&F0, (void*)&F1, (void*)&fc, (void*)&R0, (void*)&R1, (void*)&pctl, (void*)&pout};
            PeelOut hc;
            {
                // one peel at a time in the process: two grid-wide launches must
                // not each hold part of the SMs while waiting for the rest
                static std::mutex peel_mu;
                std::lock_guard<std::mutex> lock(peel_mu);
                KC_TRY(cudaLaunchCooperativeKernel((const void*)k_peel_grid, dim3((unsigned)blocks),
                                                   dim3(PEEL_THREADS), args, 0, s));
                note_launch();
                KC_TRY(cudaMemcpyAsync(&hc, pout, sizeof(PeelOut), cudaMemcpyDeviceToHost, s));
                KC_TRY(cudaMemcpyAsync(&maxdeg, words + 1, 4, cudaMemcpyDeviceToHost, s));
                KC_TRY(cudaStreamSynchronize(s));
            }
            if (hc.flags & KC_FLAG_INTERNAL)
                return fail(set_error(KC_E_INTERNAL, "k-core peel: inconsistent state after %u phases (level %u, "
                                                     "%u sub-rounds)", hc.phases, hc.max_level, hc.rounds));
            g->degeneracy = hc.max_level;
            max_key = hc.rounds;
            k_removal_key<<<grid_for((uint64_t)n * 32, 256, sms), 256, 0, s>>>(d_rp, d_ci, n, round_of, key);
            note_launch();
            KC_TRY(cudaGetLastError());
        } else {
            g->degeneracy = 0;
        }
    } else {
        KC_TRY(cudaMemcpyAsync(&max_key, words + 1, 4, cudaMemcpyDeviceToHost, s));
        KC_TRY(cudaStreamSynchronize(s));
    }

    // order: old_of_new = ids sorted by the orientation key with ties to the
    // lower id; new_of_old its inverse.  Degree: key (degree, id).
    // Degeneracy: (peel round, remaining degree when removed, id) -- inside a
    // round the vertices that had fewer neighbours left come first, as a
    // one-at-a-time min-degree peel would take them.
    KC_TRYS(dev_alloc(g->old_of_new, (size_t)n * 4 + 4));
    KC_TRYS(dev_alloc(g->new_of_old, (size_t)n * 4 + 4));
    if (degen && n > 0) {
        uint32_t* by_deg = (uint32_t*)F0;  // free after the peel
        KC_TRYS(sort_ids_by_key(key, n, maxdeg, by_deg, g->tmp, s));
        KC_TRYS(sort_ids_by_key(round_of, n, max_key, (uint32_t*)g->old_of_new.ptr, g->tmp, s, by_deg));
    } else {
        KC_TRYS(sort_ids_by_key(key, n, max_key, (uint32_t*)g->old_of_new.ptr, g->tmp, s));
    }
    k_invert<<<grid_for(n, 256, sms), 256, 0, s>>>((uint32_t*)g->old_of_new.ptr, n, (uint32_t*)g->new_of_old.ptr);
    note_launch();
    KC_TRY(cudaGetLastError());

    // out-degrees in the library numbering, then row pointers
    KC_TRYS(dev_alloc(g->row_ptr, ((size_t)n + 1) * 4));
    // rows are scanned in 16-byte quads: pad to whole quads plus one
    KC_TRYS(dev_alloc(g->col, (((size_t)g->m + 3) / 4 + 1) * 16));
    uint32_t* outdeg = (uint32_t*)F0;  // reuse
    KC_TRY(cudaMemsetAsync(outdeg, 0, (size_t)n * 4 + 4, s));
    const uint64_t fthreads = ((uint64_t)nnz + 7) / 8;
    const unsigned fblocks = (unsigned)std::max<uint64_t>(1, (fthreads + 255) / 256);
    if (nnz) {
        k_filter<0><<<fblocks, 256, 0, s>>>(d_rp, d_ci, n, nnz, (uint32_t*)g->new_of_old.ptr, outdeg, nullptr);
        note_launch();
        KC_TRY(cudaGetLastError());
    }
    uint32_t* drp = (uint32_t*)g->row_ptr.ptr;
    KC_TRYS(scan_u32(outdeg, drp, n, g->tmp, s));
    // fill (unsorted) into colbuf, then sort rows into col
    uint32_t* cursor = (uint32_t*)F1;
    KC_TRY(cudaMemcpyAsync(cursor, drp, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    if (nnz) {
        k_filter<1><<<fblocks, 256, 0, s>>>(d_rp, d_ci, n, nnz, (uint32_t*)g->new_of_old.ptr, cursor, colbuf);
        note_launch();
        KC_TRY(cudaGetLastError());
        k_sort_rows<<<grid_for((uint64_t)n * 32, ROWSORT_WARPS * 32, sms), ROWSORT_WARPS * 32, 0, s>>>(
            drp, colbuf, (uint32_t*)g->col.ptr, n);
        note_launch();
        KC_TRY(cudaGetLastError());
    }
    // d_max, out-degree histogram, root order (out-degree descending)
    KC_TRY(cudaMemsetAsync(words + 2, 0, 4, s));
    k_rowlen_max<<<grid_for(n, 256, sms), 256, 0, s>>>(drp, n, words + 2);
    note_launch();
    KC_TRY(cudaGetLastError());
    KC_TRY(cudaMemcpyAsync(&h_words[2], words + 2, 4, cudaMemcpyDeviceToHost, s));
    KC_TRY(cudaStreamSynchronize(s));
    g->d_max = h_words[2];
    unsigned* hist = (unsigned*)heavy;  // n + 1 >= d_max + 1 entries
    KC_TRY(cudaMemsetAsync(hist, 0, ((size_t)g->d_max + 1) * 4, s));
    k_outdeg_from_rowptr<<<grid_for(n, 256, sms), 256, 0, s>>>(drp, n, key, g->d_max, hist);
    note_launch();
    KC_TRY(cudaGetLastError());
    KC_TRYS(dev_alloc(g->roots, (size_t)n * 4 + 4));
    KC_TRYS(sort_ids_by_key(key, n, g->d_max, (uint32_t*)g->roots.ptr, g->tmp, s));
    std::vector<unsigned> h_hist(g->d_max + 1);
    KC_TRY(cudaMemcpyAsync(h_hist.data(), hist, h_hist.size() * 4, cudaMemcpyDeviceToHost, s));
    KC_TRY(cudaEventRecord(ev1, s));
    KC_TRY(cudaStreamSynchronize(s));
    g->outdeg_hist.assign(h_hist.begin(), h_hist.end());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    g->orient_ms = ms;
    scratch_free(work, s);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
#undef KC_TRY
#undef KC_TRYS
    return KC_OK;
}


}  // namespace kc
