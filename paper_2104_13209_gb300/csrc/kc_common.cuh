// Internal declarations shared by the CUDA translation units of libkclique.
// Nothing here is part of the public C ABI (include/kclique.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kclique.h"

#define KC_VERSION 10000

// ---------------------------------------------------------------------------
// Host-side error plumbing
// ---------------------------------------------------------------------------
namespace kc {

kc_status set_error(kc_status s, const char* fmt, ...);
void note_launch();  // counts every kernel the library launches (kc_launch_count)
void clear_error();
kc_status cuda_error(cudaError_t e, const char* what, const char* file, int line);

}  // namespace kc

#define KC_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return kc::cuda_error(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define KC_CHECK(st)                      \
    do {                                  \
        kc_status s_ = (st);              \
        if (s_ != KC_OK) return s_;       \
    } while (0)

// ---------------------------------------------------------------------------
// Device buffers owned by a handle
// ---------------------------------------------------------------------------
namespace kc {

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

kc_status dev_alloc(DevBuf& b, size_t bytes);      // (re)allocate if smaller than `bytes`
void dev_free(DevBuf& b);
// Stream-ordered scratch from a memory pool the library keeps per device
// (up to 1 GiB stays reserved between uses): working memory of one call
// that costs neither a cudaMalloc nor a device-wide cudaFree.
kc_status scratch_alloc(void** p, size_t bytes, cudaStream_t s);
void scratch_free(void* p, cudaStream_t s);

// Per-launch error word written by kernels (device) -- bit layout = KC_FLAG_*.
struct Ctl {
    unsigned long long total_lo;   // exact 128-bit count, low word
    unsigned long long total_hi;   // carries out of total_lo
    unsigned long long words;      // bitmap words intersected
    unsigned long long deadline;   // %globaltimer value after which work stops (0 = none)
    unsigned int flags;            // KC_FLAG_* bits
    unsigned int work_next;        // big-root work counter
    unsigned int work_next_small;  // small-root work counter
    unsigned int work_next_aux;    // spare counter
    unsigned int bar_count;        // grid barrier arrivals
    unsigned int bar_gen;          // grid barrier generation
    unsigned int dbg_code;         // first failed device-side bounds check (0 = none)
    unsigned int dbg_idx;          // the index it refused
};

}  // namespace kc

// The opaque handle of the public API.
struct kc_graph {
    uint32_t n = 0;
    uint64_t m = 0;             // undirected edges == DAG edges
    uint32_t d_max = 0;         // max DAG out-degree
    uint32_t degeneracy = 0xFFFFFFFFu;
    int orient = 0;
    float orient_ms = 0.f;
    int device = 0;
    int sm_count = 0;
    double time_limit_s = 0.0;  // 0 = none
    uint64_t last_work = 0;     // work units of the last synchronous count
    // DAG in the library numbering (vertex r = r-th vertex of the order)
    kc::DevBuf row_ptr;      // u32[n+1]
    kc::DevBuf col;          // u32[m]
    kc::DevBuf new_of_old;   // u32[n]
    kc::DevBuf old_of_new;   // u32[n]
    kc::DevBuf core;         // u32[n] (input numbering), degeneracy only
    kc::DevBuf roots;        // u32[n] library ids sorted by out-degree, descending
    std::vector<uint64_t> outdeg_hist;  // host: number of vertices per out-degree (d_max + 1 entries)
    // working memory for counting
    kc::DevBuf ctl;          // kc::Ctl + kernel work counters (sized by kc::ctl_bytes())
    kc::DevBuf result;       // kc_result written by the synchronous calls
    kc::DevBuf pivot_out;    // per-size counts of a pivoting run
    kc::DevBuf pv_stage;     // device staging of per-vertex counts for host outputs
    kc::DevBuf scratch;      // per-block scratch (global-memory bitmaps and stacks)
    kc::DevBuf pv;           // u64 per-vertex accumulators (library numbering) + overflow words
    kc::DevBuf tmp;          // misc temporaries
    kc::DevBuf sm_work;      // u64[SM_WORK_SLOTS]: work units per SM of the last orientation-mode count
    uint64_t device_bytes() const;
};

// ---------------------------------------------------------------------------
// Cross-unit entry points (host side)
// ---------------------------------------------------------------------------
namespace kc {

// kc_scan.cu: exclusive scan of n u32 values into out (n+1 entries, out[n] =
// total).  `tmp` is grown as needed.  Returns an error status on CUDA failure.
kc_status scan_u32(const uint32_t* in, uint32_t* out, size_t n, DevBuf& tmp, cudaStream_t s);
size_t scan_tmp_bytes(size_t n);
// Same, with caller-provided scratch of scan_tmp_bytes(n) bytes.
kc_status scan_u32_raw(const uint32_t* in, uint32_t* out, size_t n, void* tmp, cudaStream_t s);

// kc_sort.cu: stable sort of the ids 0..n-1 (or of in_ids[0..n) when given)
// by key[id], ascending; equal keys keep their input order.  out_ids receives
// the sorted ids (it must not alias in_ids).  max_key bounds the keys.
kc_status sort_ids_by_key(const uint32_t* key, uint32_t n, uint32_t max_key, uint32_t* out_ids, DevBuf& tmp,
                          cudaStream_t s, const uint32_t* in_ids = nullptr);

// kc_orient.cu
kc_status build_graph(kc_graph* g, const uint32_t* d_rp, const uint32_t* d_ci, int validate, cudaStream_t s);

// Work units per SM of an orientation-mode count (Fig. 7's load balance):
// slots indexed by %smid.
static constexpr uint32_t SM_WORK_SLOTS = 1024;

// kc_list.cu: the orientation traversal on sorted vertex lists instead of
// binary-encoded sub-graphs (the paper's comparison point), 3 <= k <=
// LIST_MAX_K.  list_launch enqueues its kernel (ctl zeroed and its deadline
// set by the caller, cursor a zeroed counter, sm_work nullable); the caller
// finalises the result.  With emitted (a zeroed counter) not null it lists
// the cliques too: the first cap of them to out (k ids each, input
// numbering; out may be null when cap is 0).  list_scratch_words: global
// scratch it takes.
static constexpr uint32_t LIST_MAX_K = 16;
kc_status list_launch(kc_graph* g, uint32_t k, bool ec, Ctl* ctl, unsigned* cursor, unsigned long long* sm_work,
                      cudaStream_t s, uint32_t* out = nullptr, unsigned long long cap = 0,
                      unsigned long long* emitted = nullptr);
// kc_count.cu: listing of the k-cliques (3 <= k <= LIST_MAX_K) by the list
// traversal; result (count, flags, status) to result_dev.
kc_status list_cliques_launch(kc_graph* g, uint32_t k, uint32_t* out, uint64_t cap, kc_result* result_dev,
                              cudaStream_t s);
size_t list_scratch_words(const kc_graph* g, uint32_t k);

// kc_count.cu
struct CountArgs {
    uint32_t k;
    int scheme;       // KC_SCHEME_VC / EC / VC_LIST / EC_LIST (resolved)
    uint32_t subwarp; // resolved group width
    int pivot;
    uint64_t* per_vertex_dev;  // input numbering, may be null
};
kc_status count_launch(kc_graph* g, const CountArgs& a, kc_result* result_dev, cudaStream_t s);
kc_status count_reserve(kc_graph* g, uint32_t k_max, int pivot, int per_vertex, cudaStream_t s);
size_t ctl_bytes();

// One query of a batched orientation-mode launch: a resident DAG (library
// numbering), the query's roots in decreasing out-degree, and its k.
struct QDesc {
    const uint32_t* rp;
    const uint32_t* col;
    const uint32_t* roots;
    uint32_t n_roots;            // entries of roots (the graph's vertices)
    uint32_t k;
    uint32_t n;                  // vertices (the k = 1 answer)
    uint32_t d_max;              // largest out-degree among the roots
    unsigned long long m;        // edges (the k = 2 answer)
    uint32_t slot;               // index of the query's kc_result in the output array
    uint32_t pad;
};

// Launch configuration of one group of a batched launch.
struct BatchConfig {
    int ec;                      // edge-centric split for the big roots
    uint32_t subwarp;            // threads per group: 1, 2, 4, 8, 16, 32
    uint32_t chunk;              // small roots a warp claims per atomic
};

// Rough cost of a query, used only to order the queries of a launch
// cheapest first: m * d_max^(min(k, 6) - 2) for 3 <= k <= d_max + 1.
inline double query_cost_estimate(unsigned long long m, uint32_t d_max, uint32_t k) {
    if (k < 3 || k > d_max + 1) return 0.0;
    double c = (double)m;
    for (uint32_t i = 2; i < (k < 6 ? k : 6); ++i) c *= (double)d_max;
    return c;
}

// Device working memory of one batched launch of nq queries.
size_t batch_ws_bytes(uint32_t nq);

// Enqueue the counts of q_dev[0, nq) (device array, one configuration) on
// stream s: working memory ws (batch_ws_bytes(nq) bytes, device, 256-byte
// aligned), results to results_dev[q.slot].  d_cap / k_max: the
// largest out-degree and k among the queries.  No allocation, no host
// synchronisation: safe to capture.
// early / done (nullable together): each query's result is also written to
// early[slot], then done[slot] = 1 after a system-scope fence, as soon as its
// last root completes (before the launch ends); host-mapped memory lets a
// host thread see results while the launch still runs.  A query that timed
// out is not published early; its results_dev entry has KC_E_TIMEOUT.
kc_status batch_launch(const QDesc* q_dev, uint32_t nq, uint32_t d_cap, uint32_t k_max, const BatchConfig& cfg,
                       void* ws, double time_limit_s, int sm_count, kc_result* results_dev, kc_result* early,
                       unsigned* done, cudaStream_t s);

// Shared memory a batched launch of this geometry needs, or 0 if it does
// not fit (bitmaps would need global memory, which batched launches do not
// take).
size_t batch_smem_bytes(uint32_t d_cap, uint32_t k_max, const BatchConfig& cfg);

// kc_deep.cu: orientation-mode counts with re-encoded small nodes, for
// k >= 5, and with per-vertex counts (pv) for k >= 3.
// deep_supported: whether the kernel takes (graph, k).  deep_plan: global
// scratch words and grid size of its launch.  deep_launch: enqueue it over
// roots[0, n_work) (roots[0, n_big) with more than 32 candidates); task_next
// and task_total hold n_big zeroed words each; pv (nullable): zeroed u64[n]
// per-vertex accumulators in the library numbering.  pv_to_input: copy them
// to out[n] in the input numbering.
bool deep_supported(const kc_graph* g, uint32_t k, bool pv);
kc_status deep_plan(const kc_graph* g, uint32_t k, bool ec, bool pv, size_t* scratch_words, int* blocks_out);
kc_status deep_launch(kc_graph* g, uint32_t k, bool ec, uint32_t n_big, uint32_t n_work, uint32_t* task_next,
                      uint32_t* task_total, uint32_t* gscratch, unsigned long long* pv, Ctl* ctl, cudaStream_t s);
kc_status pv_to_input(const kc_graph* g, const unsigned long long* pv, uint64_t* out, cudaStream_t s);

// kc_pivot.cu
// Fixed-k pivoting count into result_dev (device); per_vertex_dev: n entries
// (input numbering) or null.
kc_status count_pivot_async(kc_graph* g, uint32_t k, kc_result* result_dev, uint64_t* per_vertex_dev,
                            cudaStream_t s);
// Every size < cap by pivoting, exact below 2^128: counts_lo / counts_hi
// (host, cap entries each; counts_hi nullable), ovf128_host[j] = 1 when the
// count exceeds 2^128 - 1.  Synchronises s.
kc_status count_all_run(kc_graph* g, uint32_t cap, uint32_t pvk, uint64_t* per_vertex_dev, uint64_t* counts_lo_host,
                        uint64_t* counts_hi_host, uint8_t* ovf128_host, uint32_t* omega_host, uint32_t* flags_host,
                        cudaStream_t s);

int sm_count_of_current_device();

}  // namespace kc

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace kc {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A device-side bounds check: false (and the first failure recorded in
// c->dbg_code / dbg_idx, with KC_FLAG_INTERNAL) when idx >= bound; the
// caller then skips the access.
__device__ __forceinline__ bool in_bounds(Ctl* c, unsigned long long idx, unsigned long long bound, unsigned code) {
    if (idx < bound) return true;
    if (atomicCAS(&c->dbg_code, 0u, code) == 0u) c->dbg_idx = (unsigned)idx;
    atomicOr(&c->flags, (unsigned)KC_FLAG_INTERNAL);
    return false;
}

// Exact 128-bit accumulation of a 64-bit partial into (lo, hi).
__device__ __forceinline__ void add_u128(unsigned long long* lo, unsigned long long* hi, unsigned long long x) {
    if (x == 0) return;
    unsigned long long old = atomicAdd(lo, x);
    if (old + x < old) atomicAdd(hi, 1ull);
}

// Grid-wide barrier for cooperative launches, with a bounded wait: after
// `limit_ns` of waiting the block records KC_FLAG_TIMEOUT in *flags and
// returns false (every later barrier then returns false at once).  When dbg
// is not null a timed-out block records {block, its barrier sequence number,
// arrivals seen, generation seen, the generation it waited on} there.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen, unsigned int nblocks,
                                             unsigned int* flags, unsigned long long limit_ns,
                                             unsigned int* dbg = nullptr, unsigned int seq = 0) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = (atomicAdd(flags, 0u) & KC_FLAG_TIMEOUT) == 0;
        if (ok) {
            unsigned int g = atomicAdd(gen, 0u);
            __threadfence();
            if (atomicAdd(count, 1u) == nblocks - 1) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(gen, 1u);
            } else {
                unsigned long long t0 = globaltimer_ns();
                unsigned int spins = 0;
                while (atomicAdd(gen, 0u) == g) {
                    __nanosleep(64);
                    if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) {
                        atomicOr(flags, (unsigned)KC_FLAG_TIMEOUT);
                        if (dbg && atomicCAS(&dbg[0], 0u, 1u) == 0u) {  // the first block to give up
                            dbg[1] = blockIdx.x;
                            dbg[2] = seq;
                            dbg[3] = atomicAdd(count, 0u);
                            dbg[4] = atomicAdd(gen, 0u);
                            dbg[5] = g;
                            dbg[6] = (unsigned)(globaltimer_ns() - t0);
                        }
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace kc
#endif
