/*
 * kclique.h -- exact k-clique counting on one NVIDIA GB300 (sm_103a).
 *
 * The method is that of "Parallel K-clique Counting on GPUs" (Almasri,
 * El Hajj, Nagi, Xiong, Hwu; ICS '22):
 *   - the undirected graph is oriented into a DAG by degree or degeneracy
 *     order (Section 3.1);
 *   - every root vertex (vertex-centric) or root edge (edge-centric) gets the
 *     binary-encoded sub-graph induced by its out-neighbours (Sections 2.4,
 *     3.2 and 3.4);
 *   - a depth-first search with an explicit stack does a bitwise AND plus
 *     popcount per tree node (Fig. 2, Section 3.3), or, in pivoting mode,
 *     selects a pivot per node and counts every clique size at once (Fig. 3);
 *   - counts are reduced into exact 128-bit totals on the device and
 *     reported as uint64 plus an overflow flag.
 *
 * Conventions for every call:
 *   - Every function returns a kc_status code (KC_OK = 0).  No function
 *     aborts, exits or traps.  kc_last_error() gives a message for the last
 *     failing call on the calling host thread.
 *   - Vertex ids are uint32, counts uint64.  A graph is a CSR: row_ptr[n+1]
 *     (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz) and col_idx[nnz].
 *     nnz must be below 2^32.  The graph must be simple and undirected:
 *     symmetric, no self-loops, no duplicate entries, every row strictly
 *     ascending, every id < n.  A violation gives KC_E_INVALID_GRAPH.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it in order.  Calls that return values in
 *     host memory synchronise that stream before returning.
 *   - The caller owns every array it passes; the library copies what it keeps.
 *   - A graph handle may be used by one host thread at a time.
 */
#ifndef KCLIQUE_H
#define KCLIQUE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef int kc_status;
#define KC_OK 0
#define KC_E_INVALID_ARG 1     /* a bad argument (null pointer, k = 0, unknown enum, ...) */
#define KC_E_INVALID_GRAPH 2   /* the CSR is not a simple undirected graph */
#define KC_E_NO_MEMORY 3       /* a device or host allocation failed */
#define KC_E_OVERFLOW 4        /* a count exceeded 2^64 - 1; outputs are still written, see flags */
#define KC_E_TIMEOUT 5         /* a bounded device wait gave up; results are not valid */
#define KC_E_CUDA 6            /* a CUDA runtime call failed */
#define KC_E_INTERNAL 7        /* a device-side consistency check failed */
#define KC_E_UNSUPPORTED 8     /* a size or case beyond what the library handles */
#define KC_E_REFUSED 9         /* a serving query not admitted: its shape ran out of time before */

/* ---- enumerations ------------------------------------------------------ */
/* Orientation criterion (Section 3.1). */
#define KC_ORIENT_DEGREE 0      /* u -> v iff (deg u, u) < (deg v, v) */
#define KC_ORIENT_DEGENERACY 1  /* u -> v iff (peel round u, u) < (peel round v, v) */

/* Parallelisation scheme (Section 3.2). */
#define KC_SCHEME_AUTO 0        /* vertex-centric for k < 6, edge-centric otherwise (Section 4.5) */
#define KC_SCHEME_VC 1          /* one root vertex per work item */
#define KC_SCHEME_EC 2          /* one root edge per work item */
/* The same two splits without the binary encoding (the paper's comparison
 * point, Sections 3.4 and 4.3): candidate sets are sorted vertex lists and
 * each intersection searches the members of one list in a DAG row (binary
 * search).  Orientation traversal only, totals only (per-vertex counts give
 * KC_E_UNSUPPORTED), 3 <= k <= 16 (KC_E_UNSUPPORTED beyond); one warp per
 * root vertex (VC_LIST) or per DAG edge (EC_LIST).  Work units: membership
 * tests. */
#define KC_SCHEME_VC_LIST 3
#define KC_SCHEME_EC_LIST 4

/* Result flag bits. */
#define KC_FLAG_TOTAL_OVERFLOW 1u       /* the total exceeded 2^64 - 1 */
#define KC_FLAG_VERTEX_OVERFLOW 2u      /* some per-vertex count exceeded 2^64 - 1 */
#define KC_FLAG_TIMEOUT 4u              /* a device wait ran out of time */
#define KC_FLAG_INTERNAL 8u             /* a device-side check failed */
#define KC_FLAG_TOTAL_OVERFLOW128 16u   /* the total exceeded 2^128 - 1 (pivoting only) */

typedef struct kc_graph kc_graph;

typedef struct kc_graph_info {
    uint32_t n;            /* vertices */
    uint32_t d_max;        /* maximum out-degree of the DAG */
    uint64_t num_edges;    /* undirected edges (= DAG edges) */
    uint32_t degeneracy;   /* max core number (degeneracy orientation), else 0xFFFFFFFF */
    int32_t orient;        /* KC_ORIENT_* */
    uint64_t device_bytes; /* device memory held by the handle */
    float orient_ms;       /* device time of the orientation kernels */
} kc_graph_info;

/* Result written to DEVICE memory by the asynchronous calls. */
typedef struct kc_result {
    uint64_t total;        /* low 64 bits of the exact count */
    uint64_t total_hi;     /* high 64 bits (non-zero iff the count overflowed uint64) */
    uint32_t flags;        /* KC_FLAG_* */
    uint32_t status;       /* KC_OK or the kc_status of a device-side failure */
    uint64_t words;        /* work units: bitmap words intersected (orientation), membership tests
                              (list traversal) or tree nodes (pivoting) */
} kc_result;

/* ---- errors -------------------------------------------------------------- */
/* Message for the last failing call on this host thread ("" if none).  The
 * pointer stays valid until the next library call on this thread. */
const char* kc_last_error(void);
/* Static name of a status code ("KC_OK", ...). */
const char* kc_status_name(kc_status s);
/* Library version, major * 10000 + minor * 100 + patch. */
int kc_version(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (all threads, all devices); for accounting of device work. */
uint64_t kc_launch_count(void);

/* ---- graphs ---------------------------------------------------------------- */
/* Build a resident, oriented graph (Section 3.1: orientation on the device,
 * undesired directions dropped, row pointers rebuilt by histogram + scan).
 *   row_ptr, col_idx: the CSR, in host memory (ptrs_on_device = 0) or device
 *     memory (ptrs_on_device = 1); read during the call only.
 *   orient: KC_ORIENT_DEGREE or KC_ORIENT_DEGENERACY.
 *   validate: 1 = check that the CSR is simple and undirected (one pass on the
 *     device); 0 = trust the caller (results are undefined on a bad graph).
 *   out: receives the handle; release it with kc_graph_destroy.
 * Errors: KC_E_INVALID_ARG, KC_E_INVALID_GRAPH, KC_E_NO_MEMORY, KC_E_CUDA,
 * KC_E_TIMEOUT (the degeneracy peel's bounded grid barrier gave up). */
kc_status kc_graph_create(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t nnz,
                          int ptrs_on_device, int orient, int validate, void* stream, kc_graph** out);

/* Free the handle and its device memory.  NULL is accepted. */
kc_status kc_graph_destroy(kc_graph* g);

kc_status kc_graph_info_get(const kc_graph* g, kc_graph_info* out);

/* Time budget for the counting calls on this graph: a count still running
 * after `seconds` stops taking work, sets KC_FLAG_TIMEOUT and returns
 * KC_E_TIMEOUT (its partial count is not valid).  0 = no limit (the default).
 * The device checks the budget between work items and every few thousand
 * tree nodes, so it may be overrun by a fraction of a millisecond. */
kc_status kc_graph_set_time_limit(kc_graph* g, double seconds);

/* Work units of the last synchronous count on this graph (kc_count,
 * kc_count128, kc_count_all, kc_list_cliques): for the graph-orientation
 * traversal the 32-bit bitmap words intersected (one AND plus one popcount
 * each), for the list traversal (KC_SCHEME_VC_LIST / EC_LIST and listing) the
 * membership tests, for pivoting the search-tree nodes analysed (a pivot
 * search each). */
kc_status kc_graph_last_work(const kc_graph* g, uint64_t* units);

/* The same work units of the last orientation-mode count on this graph
 * (kc_count and kc_count_async with pivot = 0), split by the SM that did
 * them: the load balance across SMs of Section 4.4 (Fig. 7).
 *   per_sm (host, cap entries, nullable when cap = 0): per_sm[i] = units done
 *     on SM i (the %smid of the warps that did them); entries beyond the
 *     library's 1,024 slots are 0.
 *   slots_out (host): the number of slots that hold the count: the device's
 *     SM count, or more if a higher SM id reported work.
 * Reads the counters with a synchronous copy: call it after the count has
 * finished.  Before any count, or after k <= 2, every entry is 0. */
kc_status kc_graph_last_sm_work(const kc_graph* g, uint64_t* per_sm, uint32_t cap, uint32_t* slots_out);

/* Copy the oriented graph to host memory (for inspection and tests).
 *   dag_row_ptr[n+1], dag_col[num_edges]: the DAG in the library's vertex
 *     numbering, where vertex r is the r-th vertex of the orientation order,
 *     so every edge goes from a smaller to a larger id and rows ascend;
 *   new_of_old[n]: the library id of each input vertex;
 *   core[n]: core numbers (degeneracy orientation only; otherwise pass NULL).
 * Any pointer may be NULL to skip that array. */
kc_status kc_graph_export(const kc_graph* g, uint32_t* dag_row_ptr, uint32_t* dag_col, uint32_t* new_of_old,
                          uint32_t* core);

/* ---- counting ------------------------------------------------------------- */
/* Exact number of k-cliques (Sections 2.2-2.4, 3.2-3.6).
 *   k >= 1 (k = 1 gives n, k = 2 the edge count, both without a launch).
 *   pivot: 0 = graph-orientation traversal (Fig. 2); 1 = pivoting traversal
 *     restricted to size k (Fig. 3, stopping when more than k vertices are
 *     held).
 *   scheme: KC_SCHEME_AUTO / VC / EC / VC_LIST / EC_LIST.
 *   subwarp: threads per group for the big-subgraph path, 0 = automatic,
 *     else 1, 2, 4, 8, 16 or 32 (Section 3.5).
 *   total_out (host): the count modulo 2^64.
 *   per_vertex_out (nullable, n entries, host or device memory): c_k(v), the
 *     number of k-cliques containing input vertex v, modulo 2^64.  With
 *     pivot = 0 they come from the graph-orientation traversal for
 *     3 <= k <= 36 when its shared-memory geometry fits the graph; otherwise
 *     (and with pivot = 1) from the pivoting traversal restricted to size k,
 *     which then gives the total too (the counts are the same).
 *   flags_out (nullable, host): KC_FLAG_* bits.
 * Returns KC_E_OVERFLOW (with every output written) when the total or a
 * per-vertex count exceeded 2^64 - 1. */
kc_status kc_count(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, uint64_t* total_out,
                   uint64_t* per_vertex_out, uint32_t* flags_out, void* stream);

/* Same count with both 64-bit words of the exact value (the count is exact
 * below 2^128; flags as above). */
kc_status kc_count128(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, uint64_t* lo_out,
                      uint64_t* hi_out, uint32_t* flags_out, void* stream);

/* Asynchronous form: enqueue the count on `stream` and return.  The result is
 * written to result_dev (device memory) when the stream reaches it.  Device
 * working memory is taken from the handle; call kc_graph_reserve first if the
 * call will be captured into a CUDA graph (no allocation happens then).
 * per_vertex_dev: nullable, n entries of device memory, input numbering
 * (from the traversal kc_count would use for the same arguments). */
kc_status kc_count_async(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, kc_result* result_dev,
                         uint64_t* per_vertex_dev, void* stream);

/* Orientation-mode count (pivot = 0) that allocates no device memory.
 * The paper has no counterpart: this is a library interface for callers that
 * must not let a library allocate device memory, because their memory is
 * owned by another allocator (a framework's caching pool, a fixed arena) or
 * because cudaMalloc / cudaFree would synchronise a latency-critical loop.
 *   Arguments and result as kc_count_async with pivot = 0 and no per-vertex
 *   output; result_dev is device memory owned by the caller.
 *   Working memory is a fixed 4 MiB array in the library's device image,
 *   one per device: the control words and one task counter per root with
 *   more than 32 out-neighbours.  The first call on a device looks up the
 *   array's address and keeps it until the process exits (make that call
 *   before any stream capture; host threads may make it together).  A
 *   cudaDeviceReset invalidates the kept address: do not call this entry
 *   point on a device after resetting it.  Every call clears the part of
 *   the array it uses with a stream-ordered memset.
 *   Limits: returns KC_E_UNSUPPORTED when the roots with more than 32
 *   out-neighbours exceed about 1,048,500, or when d_max is so large that
 *   the per-block bitmaps do not fit in shared memory (kc_count_async then
 *   uses graph-owned global memory).
 *   Calls that overlap in time on one device (different streams or threads)
 *   share the array and race: serialise them. */
kc_status kc_count_noalloc(const kc_graph* g, uint32_t k, int scheme, uint32_t subwarp, kc_result* result_dev,
                           void* stream);

/* Pre-allocate the device working memory kc_count_async will need for
 * orientation-mode counts up to k_max (every scheme and group width), so
 * that later calls allocate nothing and can be captured into a CUDA graph.
 * The pivoting path (pivot = 1, or per-vertex counts) still allocates its
 * buffers on its first call: make one such call before a capture.  The
 * pivot and per_vertex arguments are accepted for that future use. */
kc_status kc_graph_reserve(kc_graph* g, uint32_t k_max, int pivot, int per_vertex, void* stream);

/* List the k-cliques (the paper's conclusion names listing as a use of the
 * same traversal): the orientation traversal on sorted vertex lists
 * (KC_SCHEME_VC_LIST), where every member of the last intersection closes
 * one clique and is written out instead of only counted.
 *   3 <= k <= 16 (KC_E_UNSUPPORTED otherwise, KC_E_INVALID_ARG for k = 0).
 *   cliques_dev (device memory, cap * k entries, nullable when cap = 0):
 *     clique i is cliques_dev[i k .. i k + k), k input vertex ids in the
 *     orientation order (the root first).  Which cliques fill the cap when
 *     there are more is unspecified, and so is their order.
 *   count_out (host): the number of k-cliques of the graph, also when it
 *     exceeds cap (then exactly cap cliques are written).
 * Synchronises the stream.  The time limit of the graph applies
 * (KC_E_TIMEOUT; the written cliques are then a subset).  Work units of the
 * call: membership tests (kc_graph_last_work, kc_graph_last_sm_work). */
kc_status kc_list_cliques(kc_graph* g, uint32_t k, uint32_t* cliques_dev, uint64_t cap, uint64_t* count_out,
                          void* stream);

/* Every clique size at once by pivoting (Fig. 3, Section 2.3).
 *   counts (host, cap entries): counts[j] = number of j-cliques modulo 2^64,
 *     counts[0] = 1 by convention, entries beyond the clique number are 0.
 *   overflow (host, nullable, cap entries): 1 where counts[j] exceeded 2^64-1.
 *   omega_out (nullable): the clique number.
 *   per_vertex_k, per_vertex_out: if per_vertex_k > 0 and per_vertex_out is
 *     not NULL, per_vertex_out[v] = c_{per_vertex_k}(v) modulo 2^64 (n entries,
 *     host or device memory).
 * Returns KC_E_OVERFLOW (outputs written) when any reported count overflowed. */
kc_status kc_count_all(kc_graph* g, uint64_t* counts, uint8_t* overflow, uint32_t cap, uint32_t* omega_out,
                       uint32_t per_vertex_k, uint64_t* per_vertex_out, void* stream);

/* kc_count_all with exact counts below 2^128 (Fig. 3's leaf sums C(q, j - h)
 * carried in 128-bit arithmetic; Table 1's counts reach 5.4e18 and the
 * middle sizes of dense graphs pass 2^64).
 *   counts_lo, counts_hi (host, cap entries each): the low and high 64-bit
 *     words of c_j; counts_lo[0] = 1.
 *   overflow (host, nullable, cap entries): 1 where c_j exceeded 2^128 - 1
 *     (the words are then not exact).
 *   omega_out, per_vertex_k, per_vertex_out: as kc_count_all (per-vertex
 *     counts stay 64-bit, flagged beyond 2^64 - 1).
 * Returns KC_E_OVERFLOW (outputs written) when a count exceeded 2^128 - 1 or
 * a per-vertex count exceeded 2^64 - 1. */
kc_status kc_count_all128(kc_graph* g, uint64_t* counts_lo, uint64_t* counts_hi, uint8_t* overflow, uint32_t cap,
                          uint32_t* omega_out, uint32_t per_vertex_k, uint64_t* per_vertex_out, void* stream);

/* ---- batched counts over many small graphs -------------------------------
 * The paper counts one graph at a time; these calls serve workloads of
 * thousands of small graphs (ego networks, per-query subgraphs) with uneven
 * k, counted by the orientation traversal (Fig. 2) in persistent launches
 * that span every query.  A query's graph is oriented as a block of one
 * union graph (Section 3.1); its count is exact (128-bit) like kc_count128. */
typedef struct kc_batch kc_batch;
typedef struct kc_batch_exec kc_batch_exec;

/* Launch configuration chosen for one (out-degree class, k) bucket.
 * dclass: 0 for largest out-degree <= 32, c for <= 32 * 2^c (c <= 5), 6
 * beyond.  scheme: KC_SCHEME_VC or KC_SCHEME_EC for the roots with more than
 * 32 candidates (Section 3.2); subwarp: threads per group (Section 3.5);
 * chunk: roots a warp claims per atomic among the small roots (the work
 * tile); ms: the measured time of the bucket's sample. */
typedef struct kc_tune_entry {
    uint32_t dclass;
    uint32_t k;
    int32_t scheme;
    uint32_t subwarp;
    uint32_t chunk;
    float ms;
} kc_tune_entry;

#define KC_TUNE_MAX 256
typedef struct kc_tune {
    uint32_t n;
    kc_tune_entry e[KC_TUNE_MAX];
} kc_tune;

/* Build a batch from a block-diagonal CSR: graph g owns the vertices
 * [graph_offsets[g], graph_offsets[g + 1]) (host array, num_graphs + 1
 * entries, 0 first and n last) and no edge may leave that range
 * (KC_E_INVALID_GRAPH when validate is set).  The other arguments are those
 * of kc_graph_create; the caller keeps its arrays. */
kc_status kc_batch_create(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t nnz,
                          const uint32_t* graph_offsets, uint32_t num_graphs, int ptrs_on_device, int orient,
                          int validate, void* stream, kc_batch** out);
kc_status kc_batch_destroy(kc_batch* b);

/* Vertices, edges and largest DAG out-degree of graph `graph` (outputs
 * nullable). */
kc_status kc_batch_graph_info(const kc_batch* b, uint32_t graph, uint32_t* n, uint64_t* m, uint32_t* d_max);

/* Time limit of each launch (seconds, 0 = none); a launch that runs out
 * marks its queries KC_E_TIMEOUT in their results. */
kc_status kc_batch_set_time_limit(kc_batch* b, double seconds);

/* Count nq queries: query i is (graph_ids[i], ks[i]) (host arrays, ks[i] >=
 * 1).  Results go to results_dev[i] (device memory, nq entries): total and
 * total_hi (exact below 2^128), KC_FLAG_* flags, status KC_OK or
 * KC_E_TIMEOUT.  tune (nullable): configuration per bucket; buckets it does
 * not list take the paper's guideline (Section 4.5).  Queries that share a
 * launch configuration form one launch, whose roots must number fewer than
 * 2^31 (KC_E_UNSUPPORTED otherwise).  Stream-ordered; the call may wait for
 * its own previous call's descriptor copy and may allocate, so use
 * kc_batch_capture for CUDA-graph replay. */
kc_status kc_batch_count(kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq,
                         kc_result* results_dev, const kc_tune* tune, void* stream);

/* Autotuner: for every (out-degree class, k) bucket of the given queries,
 * time each candidate configuration (VC / EC, 2 / 4 / 8 / 32 threads per
 * group, 4 / 32 small roots per claim) on up to `sample` of the bucket's
 * queries (0 = 256) and keep the fastest in tune_out.  Then time the
 * assembled table on all the queries against uniform configurations (one
 * launch for every bucket) and keep whichever is fastest.  Synchronises the
 * stream. */
kc_status kc_batch_tune(kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq, uint32_t sample,
                        kc_tune* tune_out, void* stream);

/* Capture the launches of kc_batch_count for these queries into a CUDA
 * graph (descriptors staged in memory the executable owns).  Every
 * kc_batch_exec_launch then replays them on `stream`, writing results_dev,
 * which must stay valid while the executable exists. */
kc_status kc_batch_capture(kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq,
                           kc_result* results_dev, const kc_tune* tune, kc_batch_exec** out);
kc_status kc_batch_exec_launch(kc_batch_exec* e, void* stream);
kc_status kc_batch_exec_destroy(kc_batch_exec* e);

/* ---- serving ----------------------------------------------------------------
 * No counterpart in the paper.  A server keeps oriented graphs resident and
 * answers count queries (graph, k, pivot) from a worker thread of its own:
 * orientation-mode queries that arrive while others run are packed, up to
 * max_batch at a time, into persistent batched launches on `slots` streams
 * that overlap on the device (each on SMs / slots of the GPU), and each
 * query's result is served as soon as its last root completes.  Pivot-mode
 * queries (Fig. 3, fixed k), and orientation queries whose bitmaps exceed
 * shared memory, take a slot each on the graph's own path, one per graph at
 * a time.  Counts are those of kc_count / kc_count128. */
typedef struct kc_server kc_server;

typedef struct kc_server_result {
    uint64_t total;        /* count modulo 2^64 */
    uint64_t total_hi;     /* high word (orientation mode; exact below 2^128) */
    uint32_t flags;        /* KC_FLAG_* */
    int32_t status;        /* KC_OK, KC_E_TIMEOUT, ... */
    uint32_t graph_id;
    uint32_t k;
    int32_t pivot;
    uint32_t launch;       /* the launch that served it (1, 2, ...) */
    double t_submit_ms;    /* times since the server's creation (host clock) */
    double t_admit_ms;
    double t_done_ms;
} kc_server_result;

/* One launch in flight at a time, one query per launch (the plain baseline). */
#define KC_SERVER_SERIAL 1
/* The server picks the traversal of every query; the query's own pivot
 * flag is then only recorded (the count is the same either way).  With a
 * time limit set, kc_server_add_graph first measures the graph's cost
 * profile on the SM share a query gets: the orientation traversal at
 * k = 3, 4, ... (up to 16 and d_max + 1), each under the time limit, until
 * one runs out of it (every larger k is then taken as expensive); if one
 * did, the pivot traversal over every k, and if that ran out too, the pivot
 * traversal at that k and up, until one runs out (the larger k are then
 * expensive by pivoting too).  Counts of the profile are not kept.  A query takes
 * the orientation traversal unless the profile found it expensive at its
 * k, then pivoting unless that was found expensive too.  Without a profile
 * (no time limit when the graph was added): the paper's guideline (Section
 * 4.5), orientation below k = 7 and pivoting from k = 7. */
#define KC_SERVER_AUTO_TRAVERSAL 2
/* Admission control: a query is refused at once (KC_E_REFUSED), instead of
 * waiting for a slot and timing out, when its shape (graph, k, traversal)
 * is expensive: the graph's cost profile ran out of the time limit there,
 * or an earlier query of that shape did. */
#define KC_SERVER_REFUSE_EXPENSIVE 4

/* hbm_budget: device bytes the server may keep resident (slots and graphs);
 * a graph that would exceed it is refused with KC_E_NO_MEMORY.
 * max_batch >= 1 queries per batched launch; slots >= 1 launches in flight.
 * flags: 0 or a combination of KC_SERVER_SERIAL (one launch at a time, in
 *   arrival order: the plain baseline), KC_SERVER_AUTO_TRAVERSAL and
 *   KC_SERVER_REFUSE_EXPENSIVE.  The calling thread's current
 * device is the server's. */
kc_status kc_server_create(size_t hbm_budget, uint32_t max_batch, uint32_t slots, int flags, kc_server** out);

/* Add a graph (arguments as kc_graph_create; the server orients and keeps
 * it); *graph_id receives its id (0, 1, ...). */
kc_status kc_server_add_graph(kc_server* s, const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n,
                              uint64_t nnz, int ptrs_on_device, int orient, int validate, uint32_t* graph_id);

/* Time limit of each launch in seconds (0 = none): a query not finished by
 * then is answered with KC_E_TIMEOUT; the others of its launch are not
 * affected. */
kc_status kc_server_set_time_limit(kc_server* s, double seconds);

/* Queue a query; *ticket identifies it.  Thread-safe. */
kc_status kc_server_submit(kc_server* s, uint32_t graph_id, uint32_t k, int pivot, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: no limit) for a query; KC_OK with *out
 * filled when it is done (its own status is out->status), KC_E_TIMEOUT if
 * it is not done yet.  Thread-safe. */
kc_status kc_server_poll(kc_server* s, uint64_t ticket, kc_server_result* out, int timeout_ms);

/* Launches so far, queries served, resident device bytes (nullable). */
kc_status kc_server_stats(kc_server* s, uint64_t* launches, uint64_t* served, uint64_t* resident_bytes);

/* Admission state of a shape: *state = 0 unknown, 1 finished within the
 * time limit when the graph was profiled (*ms: its wall time, if ms is not
 * NULL), 2 expensive (its profile or a query of it ran out of the limit).
 * k >= 1; k beyond 127 shares the entry of 127. */
kc_status kc_server_shape(kc_server* s, uint32_t graph_id, uint32_t k, int pivot, int* state, double* ms);

/* Stop the worker after the launches in flight and free everything. */
kc_status kc_server_destroy(kc_server* s);

#ifdef __cplusplus
}
#endif

#endif /* KCLIQUE_H */
