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

#include "kc_common.cuh"

namespace kc {

static constexpr uint32_t UNSET = 0xFFFFFFFFu;
static constexpr uint32_t HEAVY_DEG = 4096;
static constexpr unsigned long long PEEL_BARRIER_LIMIT_NS = 4000000000ull;  // 4 s

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
// Level-synchronous k-core peeling (cooperative launch).  At level L every
// remaining vertex of degree <= L is removed in sub-rounds: removing a
// frontier decrements the degrees of its remaining neighbours, and a
// neighbour whose degree falls to L joins the next frontier.  A vertex's
// orientation key is its sub-round index; its core number is L.  A vertex
// removed at level L had at most L remaining neighbours, so the DAG that
// orients edges by (round, id) has out-degree <= degeneracy.
// Each level's scan reads only the vertices still remaining and writes the
// survivors to the other list, and a vertex is marked removed when it
// enters a frontier (two grid barriers per sub-round).  Decrements from its
// own entry round still reach it, so its final degree is its remaining
// degree at removal (the second orientation key, k_removal_degree).
// ---------------------------------------------------------------------------
struct PeelCtl {
    unsigned fcount[2];
    unsigned rcount[2];     // lengths of the remaining-vertex lists being built
    unsigned minrem[2];
    unsigned hcount[2];     // heavy-list length, by round parity
    unsigned bar_count;
    unsigned bar_gen;
    unsigned flags;
    unsigned max_level;
    unsigned rounds;
    unsigned dbg[8];        // where a timed-out barrier gave up (see grid_barrier)
    unsigned seq_max;       // highest barrier sequence number reached by any block
    unsigned seq_min_done;  // lowest sequence number among blocks that finished
    unsigned mismatch[6];   // first disagreement between blocks on a frontier size (see log_nf)
};

// Every block logs the frontier size it read right after barrier number
// `seq` (a ring of 65536 (seq, size) entries).  A block that reads a different
// size than the first logger of the same barrier records the disagreement in
// c->mismatch; the host reports it after the kernel (KC_E_INTERNAL).  Nothing
// here changes the control flow of the kernel.
static constexpr uint32_t NF_LOG = 65536;
__device__ __forceinline__ void log_nf(PeelCtl* c, unsigned long long* nf_log, uint32_t nf, uint32_t seq) {
    if (threadIdx.x != 0) return;
    unsigned long long want = ((unsigned long long)seq << 32) | nf;
    unsigned long long* e = &nf_log[seq & (NF_LOG - 1)];
    unsigned long long cur = atomicAdd(e, 0ull);
    for (int tries = 0; tries < 8; ++tries) {
        if ((uint32_t)(cur >> 32) == seq) {
            if ((uint32_t)cur != nf && atomicCAS(&c->mismatch[0], 0u, 1u) == 0u) {
                c->mismatch[1] = seq;
                c->mismatch[2] = (uint32_t)cur;
                c->mismatch[3] = nf;
                c->mismatch[4] = blockIdx.x;
            }
            return;
        }
        unsigned long long prev = atomicCAS(e, cur, want);
        if (prev == cur) return;
        cur = prev;
    }
}

// All 32 lanes call; lanes with pred append val to buf (capacity cap).  A
// push beyond the capacity is dropped and recorded as KC_FLAG_INTERNAL.
__device__ __forceinline__ void warp_push(bool pred, uint32_t val, uint32_t* buf, unsigned* cnt, uint32_t cap,
                                          unsigned* flags) {
    unsigned b = __ballot_sync(0xffffffffu, pred);
    if (b == 0) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(b) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    uint32_t pos = base + __popc(b & lanemask_lt());
    if (pred) {
        if (pos < cap) __stcg(&buf[pos], val);
        else atomicOr(flags, (unsigned)KC_FLAG_INTERNAL);
    }
}

// Control words written by other SMs are read with an atomic (served by L2,
// never by a stale L1 line) by thread 0 and broadcast to the block.
__device__ __forceinline__ unsigned block_read(unsigned* p) {
    __shared__ unsigned s_val;
    __syncthreads();
    if (threadIdx.x == 0) s_val = atomicAdd(p, 0u);
    __syncthreads();
    return s_val;
}

// deg[] and round_of[] change under other SMs between grid barriers: read
// them from L2 (ld.global.cg) so no stale L1 line is ever used.
// A neighbour w of a vertex removed in round `round` loses one degree unless
// it was removed before (round_of[w] <= round).  The decrement that brings
// it to `level` pushes it into the next frontier and marks it removed in
// round + 1 at once; decrements by other vertices of this round still
// reach it, so that its final degree is its remaining degree at removal.
__device__ __forceinline__ void peel_neighbour(const uint32_t* ci, uint32_t j, bool in_range, uint32_t level,
                                               uint32_t round, int* deg, uint32_t* round_of, uint32_t* core,
                                               uint32_t* Fn, unsigned* fcn, uint32_t n, unsigned* flags) {
    bool push = false;
    uint32_t w = 0;
    if (in_range) {
        w = ci[j];
        const uint32_t r = w < n ? __ldcg(&round_of[w]) : 0u;
        if (w < n && (r == UNSET || r == round + 1)) {
            int old = atomicSub(&deg[w], 1);
            push = (old == (int)level + 1);
            if (push) {
                __stcg(&round_of[w], round + 1);
                core[w] = level;
            }
        }
    }
    warp_push(push, w, Fn, fcn, n, flags);
}

__device__ __forceinline__ bool peel_barrier(PeelCtl* c, uint32_t nb, uint32_t& seq) {
    // every thread publishes its own writes of the phase before arriving
    __threadfence();
    ++seq;
    if (threadIdx.x == 0) atomicMax(&c->seq_max, seq);
    return grid_barrier(&c->bar_count, &c->bar_gen, nb, &c->flags, PEEL_BARRIER_LIMIT_NS, c->dbg, seq);
}

__global__ void __launch_bounds__(256) k_peel(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci,
                                              uint32_t n, int* deg, uint32_t* round_of, uint32_t* core, uint32_t* F0,
                                              uint32_t* F1, uint32_t* heavy, PeelCtl* c, unsigned long long* nf_log,
                                              uint32_t* R0, uint32_t* R1) {
    const uint32_t nb = gridDim.x;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
    uint32_t* F[2] = {F0, F1};
    uint32_t* R[2] = {R0, R1};  // remaining vertices: each scan reads one list and writes the next
    uint32_t level = 0, round = 0, remaining = n;
    int cur = 0;
    int rc = 0;                 // the list the next scan reads (the first scan reads every vertex)
    uint32_t rn = n;            // its length
    bool all = true;
    uint32_t it = 0;
    uint32_t seq = 0;
    while (remaining > 0) {
        // scan: collect remaining vertices with degree <= level, keep the
        // others in the next remaining list, and track the smallest degree
        // above the level
        unsigned* mr = &c->minrem[it & 1];
        const int rx = rc ^ 1;
        uint32_t local_min = UNSET;
        for (uint32_t base = gwarp * 32; base < rn; base += nwarps * 32) {
            const uint32_t idx = base + lane;
            uint32_t v = 0;
            bool take = false, keep = false;
            if (idx < rn) {
                v = all ? idx : __ldcg(&R[rc][idx]);
                if (__ldcg(&round_of[v]) == UNSET) {
                    int d = __ldcg(&deg[v]);
                    if (d <= (int)level) {
                        take = true;
                        __stcg(&round_of[v], round);  // removed in this level's first round
                        core[v] = level;
                    } else {
                        keep = true;
                        local_min = min(local_min, (uint32_t)d);
                    }
                }
            }
            warp_push(take, v, F[cur], &c->fcount[cur], n, &c->flags);
            warp_push(keep, v, R[rx], &c->rcount[rx], n, &c->flags);
        }
        for (int o = 16; o > 0; o >>= 1) local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
        if (lane == 0 && local_min != UNSET) atomicMin(mr, local_min);
        if (!peel_barrier(c, nb, seq)) return;
        if (gtid == 0) atomicExch(&c->minrem[(it + 1) & 1], UNSET);
        ++it;
        {
            // the list just written is the next one to read; the counter of the
            // one just read is free (every block read it before this barrier)
            const uint32_t rn_new = block_read(&c->rcount[rx]);
            if (gtid == 0) atomicExch(&c->rcount[rc], 0u);
            rc = rx;
            rn = min(rn_new, n);
            all = false;
        }
        uint32_t nf = block_read(&c->fcount[cur]);
        log_nf(c, nf_log, nf, seq);
        if (nf > n || (block_read(&c->flags) & KC_FLAG_INTERNAL)) return;  // recorded in flags
        if (nf == 0) {
            uint32_t m = block_read(mr);
            if (m == UNSET || m <= level) {  // cannot happen on a consistent state
                if (gtid == 0) atomicOr(&c->flags, (unsigned)KC_FLAG_INTERNAL);
                return;
            }
            level = m;
            if (!peel_barrier(c, nb, seq)) return;
            continue;
        }
        while (nf > 0) {
            // the frontier F[cur] is already marked removed in `round`
            const int nxt = cur ^ 1;
            if (gtid == 0) atomicMax(&c->max_level, level);
            // Counter resets sit between two grid barriers and the next use of
            // the counter: the other parity's heavy counter (last read in the
            // previous round's heavy phase, next written in the next round's
            // light phase) is cleared here, and this frontier's counter in the
            // heavy phase below.
            if (gtid == 0) atomicExch(&c->hcount[(round + 1) & 1], 0u);
            // light frontier vertices: one warp each
            for (uint32_t i = gwarp; i < nf; i += nwarps) {
                uint32_t u = __ldcg(&F[cur][i]);
                uint32_t b = rp[u], e = rp[u + 1];
                if (e - b > HEAVY_DEG) {
                    if (lane == 0) {
                        uint32_t hpos = atomicAdd(&c->hcount[round & 1], 1u);
                        if (hpos < n) __stcg(&heavy[hpos], u);
                        else atomicOr(&c->flags, (unsigned)KC_FLAG_INTERNAL);
                    }
                    continue;
                }
                for (uint32_t j0 = b; j0 < e; j0 += 32)
                    peel_neighbour(ci, j0 + lane, j0 + lane < e, level, round, deg, round_of, core, F[nxt],
                                   &c->fcount[nxt], n, &c->flags);
            }
            if (!peel_barrier(c, nb, seq)) return;
            // heavy frontier vertices: the whole grid on each.  Every block
            // read nf before the light barrier: this frontier's counter is free.
            if (gtid == 0) atomicExch(&c->fcount[cur], 0u);
            uint32_t hc = min(block_read(&c->hcount[round & 1]), n);
            for (uint32_t h = 0; h < hc; ++h) {
                uint32_t u = __ldcg(&heavy[h]);
                uint32_t b = rp[u], e = rp[u + 1];
                for (uint32_t j0 = b + gwarp * 32; j0 < e; j0 += nwarps * 32)
                    peel_neighbour(ci, j0 + lane, j0 + lane < e, level, round, deg, round_of, core, F[nxt],
                                   &c->fcount[nxt], n, &c->flags);
            }
            if (!peel_barrier(c, nb, seq)) return;
            remaining -= nf;
            ++round;
            uint32_t nf_next = block_read(&c->fcount[nxt]);
            log_nf(c, nf_log, nf_next, seq);
            if (nf_next > n || (block_read(&c->flags) & KC_FLAG_INTERNAL)) return;  // recorded in flags
            cur = nxt;
            nf = nf_next;
        }
        // the next scan pushes into the counter every block just read as empty
        if (!peel_barrier(c, nb, seq)) return;
        ++level;
    }
    if (gtid == 0) c->rounds = round;
    if (threadIdx.x == 0) atomicMin(&c->seq_min_done, seq);
}

// ---------------------------------------------------------------------------
// Relabel + filter
// ---------------------------------------------------------------------------
// remaining degree of every vertex when it was removed (its final degree)
__global__ void k_removal_degree(const int* __restrict__ deg, uint32_t n, uint32_t* __restrict__ atrem) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) atrem[v] = (uint32_t)max(0, deg[v]);
}

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

__global__ void k_outdeg_from_rowptr(const uint32_t* __restrict__ rp, uint32_t n, uint32_t* __restrict__ key,
                                     uint32_t dmax, unsigned* __restrict__ hist) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        uint32_t d = rp[r + 1] - rp[r];
        key[r] = dmax - d;
        atomicAdd(&hist[d], 1u);
    }
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
    DevBuf work;
    size_t wbytes = al(sizeof(PeelCtl)) + al(64) + 8 * al((size_t)n * 4 + 4) + al(((size_t)nnz / 2 + 1) * 4) +
                    al((size_t)NF_LOG * 8);
    kc_status st = dev_alloc(work, wbytes);
    if (st != KC_OK) return st;
    char* p = (char*)work.ptr;
    PeelCtl* ctl = (PeelCtl*)p; p += al(sizeof(PeelCtl));
    unsigned* words = (unsigned*)p; p += al(64);            // [0] validate flags, [1] max key, [2] d_max
    uint32_t* key = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    int* deg = (int*)p; p += al((size_t)n * 4 + 4);
    uint32_t* round_of = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* F0 = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* F1 = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* heavy = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* R0 = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* R1 = (uint32_t*)p; p += al((size_t)n * 4 + 4);
    uint32_t* colbuf = (uint32_t*)p; p += al(((size_t)nnz / 2 + 1) * 4);
    unsigned long long* nf_log = (unsigned long long*)p;

    auto fail = [&](kc_status e) {
        dev_free(work);
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

    KC_TRY(cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), s));
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
    if (degen) {
        KC_TRYS(dev_alloc(g->core, (size_t)n * 4 + 4));
        if (n > 0) {
            int bps = 0;
            KC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_peel, 256, 0));
            if (bps < 1) return fail(set_error(KC_E_INTERNAL, "peel kernel cannot be resident"));
            unsigned blocks = (unsigned)std::min<uint64_t>((uint64_t)bps * sms, std::max<uint64_t>(1, ((uint64_t)n + 255) / 256));
            KC_TRY(cudaMemsetAsync(ctl->minrem, 0xFF, sizeof(ctl->minrem), s));
            KC_TRY(cudaMemsetAsync(&ctl->seq_min_done, 0xFF, sizeof(unsigned), s));
            const uint32_t* a_rp = d_rp;
            const uint32_t* a_ci = d_ci;
            uint32_t a_n = n;
            uint32_t* a_core = (uint32_t*)g->core.ptr;
            KC_TRY(cudaMemsetAsync(nf_log, 0xFF, (size_t)NF_LOG * 8, s));
            void* args[] = {(void*)&a_rp, (void*)&a_ci, (void*)&a_n, (void*)&deg, (void*)&round_of,
                            (void*)&a_core, (void*)&F0, (void*)&F1, (void*)&heavy, (void*)&ctl, (void*)&nf_log,
                            (void*)&R0, (void*)&R1};
            KC_TRY(cudaLaunchCooperativeKernel((const void*)k_peel, dim3(blocks), dim3(256), args, 0, s));
            note_launch();
            PeelCtl hc;
            KC_TRY(cudaMemcpyAsync(&hc, ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
            KC_TRY(cudaStreamSynchronize(s));
            if (hc.flags & KC_FLAG_TIMEOUT)
                return fail(set_error(KC_E_TIMEOUT,
                                      "k-core peel: a grid barrier wait ran out of time (blocks %u; gave up: block %u "
                                      "seq %u arrivals %u gen %u waited-gen %u after %u ns; max seq %u, min finished "
                                      "seq %u, rounds %u, level %u, flags %u; mismatch %u after barrier %u %u/%u block %u %u)",
                                      blocks, hc.dbg[1], hc.dbg[2], hc.dbg[3], hc.dbg[4], hc.dbg[5], hc.dbg[6],
                                      hc.seq_max, hc.seq_min_done, hc.rounds, hc.max_level, hc.flags, hc.mismatch[0],
                                      hc.mismatch[1], hc.mismatch[2], hc.mismatch[3], hc.mismatch[4], hc.mismatch[5]));
            if ((hc.flags & KC_FLAG_INTERNAL) || hc.mismatch[0])
                return fail(set_error(KC_E_INTERNAL,
                                      "k-core peel: inconsistent state (blocks %u; flags %u; frontier-size disagreement "
                                      "%u: after barrier %u first %u then %u by block %u; rounds %u level %u)",
                                      blocks, hc.flags, hc.mismatch[0], hc.mismatch[1], hc.mismatch[2], hc.mismatch[3],
                                      hc.mismatch[4], hc.rounds, hc.max_level));
            g->degeneracy = hc.max_level;
            max_key = hc.rounds;
            k_removal_degree<<<grid_for(n, 256, sms), 256, 0, s>>>(deg, n, key);
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
        unsigned maxdeg = 0;
        KC_TRY(cudaMemcpyAsync(&maxdeg, words + 1, 4, cudaMemcpyDeviceToHost, s));
        KC_TRY(cudaStreamSynchronize(s));
        uint32_t* by_deg = F0;  // free after the peel
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
    uint32_t* outdeg = F0;  // reuse
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
    uint32_t* cursor = F1;
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
    dev_free(work);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
#undef KC_TRY
#undef KC_TRYS
    return KC_OK;
}


}  // namespace kc
