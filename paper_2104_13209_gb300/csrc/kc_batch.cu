// Batched counts over many small graphs (include/kclique.h, kc_batch_*).
//
// The graphs arrive as one block-diagonal CSR (graph g owns the vertex range
// [off[g], off[g + 1]) and no edge leaves it).  The union is oriented once,
// as any graph (an order of the union restricted to one graph is an order of
// that graph, so every graph's DAG is the union's restricted to it), and the
// union's roots are regrouped by graph, each group in decreasing out-degree.
// A query (graph, k) is then a descriptor over the union's arrays; queries
// with the same launch configuration go to one persistent launch
// (batch_launch in kc_count.cu).  The configuration of a query comes from a
// tuning table keyed by (out-degree class, k), filled by kc_batch_tune from
// timed trials, or else from the paper's guideline (Section 4.5).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "kc_common.cuh"

struct kc_batch {
    kc_graph* g = nullptr;                  // the oriented union
    uint32_t ng = 0;
    std::vector<uint32_t> off;              // graph vertex offsets, ng + 1
    std::vector<unsigned long long> m;      // edges per graph
    std::vector<uint32_t> dmax;             // largest out-degree per graph
    kc::DevBuf roots;                       // union roots grouped by graph
    kc::DevBuf ws;                          // descriptors + per-group working memory
    void* stage = nullptr;                  // pinned host staging of the descriptors
    size_t stage_bytes = 0;
    cudaEvent_t staged = nullptr;           // the last copy out of the staging buffer
    bool staged_pending = false;
};

struct kc_batch_exec {
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;         // kernel launches inside the graph
    kc::DevBuf ws;
    void* stage = nullptr;
};

namespace kc {

__global__ void k_check_blocks(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ ci,
                               const uint32_t* __restrict__ off, uint32_t ng, uint32_t n, unsigned* bad) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t lo = 0, hi = ng;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid + 1] <= v) lo = mid + 1; else hi = mid;
        }
        const uint32_t a = off[lo], b = off[lo + 1];
        for (uint32_t j = rp[v]; j < rp[v + 1]; ++j)
            if (ci[j] < a || ci[j] >= b) atomicExch(bad, 1u);
    }
}

// graph of every library vertex (through the input numbering)
__global__ void k_graph_of(const uint32_t* __restrict__ old_of_new, const uint32_t* __restrict__ off, uint32_t ng,
                           uint32_t n, uint32_t* __restrict__ gid) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t o = old_of_new[v];
        uint32_t lo = 0, hi = ng;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid + 1] <= o) lo = mid + 1; else hi = mid;
        }
        gid[v] = lo;
    }
}

// per graph: edge count (sum of out-degrees) and largest out-degree
__global__ void k_graph_sizes(const uint32_t* __restrict__ rp, const uint32_t* __restrict__ roots,
                              const uint32_t* __restrict__ off, unsigned long long* __restrict__ m,
                              uint32_t* __restrict__ dmax) {
    const uint32_t g = blockIdx.x;
    const uint32_t a = off[g], b = off[g + 1];
    unsigned long long s = 0;
    uint32_t mx = 0;
    for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const uint32_t r = roots[i], d = rp[r + 1] - rp[r];
        s += d;
        mx = max(mx, d);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __shared__ unsigned long long ss[32];
    __shared__ uint32_t sm[32];
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (uint32_t w = 1; w < blockDim.x / 32; ++w) {
            s += ss[w];
            mx = max(mx, sm[w]);
        }
        m[g] = s;
        dmax[g] = mx;
    }
}

// out-degree class of a query's graph (the tuning table's first key)
static uint32_t dclass_of(uint32_t dmax) {
    uint32_t c = 0, cap = 32;
    while (c < 6 && dmax > cap) {
        ++c;
        cap <<= 1;
    }
    return c;
}

// the paper's guideline (Section 4.5): vertex-centric below k = 6,
// edge-centric from there; narrow groups for narrow bitmaps
static BatchConfig prior_config(uint32_t dclass, uint32_t k) {
    BatchConfig c;
    c.ec = k >= 6;
    c.subwarp = dclass <= 3 ? 4 : 8;
    c.chunk = 16;
    return c;
}

static BatchConfig config_for(const kc_tune* t, uint32_t dclass, uint32_t k) {
    if (t)
        for (uint32_t i = 0; i < t->n && i < KC_TUNE_MAX; ++i)
            if (t->e[i].dclass == dclass && t->e[i].k == k) {
                BatchConfig c;
                c.ec = t->e[i].scheme == KC_SCHEME_EC;
                c.subwarp = t->e[i].subwarp;
                c.chunk = t->e[i].chunk ? t->e[i].chunk : 1;
                return c;
            }
    return prior_config(dclass, k);
}

// One planned launch: a run of descriptors sharing a configuration.
struct Group {
    BatchConfig cfg;
    uint32_t first, count, d_cap, k_max;
    size_t ws_off;
};

struct Plan {
    std::vector<QDesc> q;      // descriptors, grouped
    std::vector<Group> groups;
    size_t ws_bytes = 0;       // descriptors + every group's working memory
};

static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

static kc_status make_plan(const kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq,
                           const kc_tune* tune, const BatchConfig* force, Plan& P) {
    struct Item {
        std::tuple<int, uint32_t, uint32_t> key;
        double cost;
        uint32_t idx;
    };
    std::vector<Item> items(nq);
    for (uint32_t i = 0; i < nq; ++i) {
        const uint32_t g = graph_ids[i], k = ks[i];
        if (g >= b->ng) return set_error(KC_E_INVALID_ARG, "query %u: graph %u out of range (%u graphs)", i, g, b->ng);
        if (k == 0) return set_error(KC_E_INVALID_ARG, "query %u: k must be >= 1", i);
        if (k > 68) return set_error(KC_E_UNSUPPORTED, "query %u: orientation traversal supports k <= 68", i);
        const BatchConfig c = force ? *force : config_for(tune, dclass_of(b->dmax[g]), k);
        items[i].key = std::make_tuple(c.ec, c.subwarp, c.chunk);
        items[i].cost = query_cost_estimate(b->m[g], b->dmax[g], k);
        items[i].idx = i;
    }
    // launches by configuration; inside one, cheapest queries first
    std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        return x.key != y.key ? x.key < y.key : x.cost < y.cost;
    });
    P.q.resize(nq);
    P.groups.clear();
    size_t off_ws = al((size_t)nq * sizeof(QDesc) + 16);
    for (uint32_t i = 0; i < nq; ++i) {
        const uint32_t qi = items[i].idx, g = graph_ids[qi];
        QDesc& D = P.q[i];
        D.rp = (const uint32_t*)b->g->row_ptr.ptr;
        D.col = (const uint32_t*)b->g->col.ptr;
        D.roots = (const uint32_t*)b->roots.ptr + b->off[g];
        D.n_roots = b->off[g + 1] - b->off[g];
        D.k = ks[qi];
        D.n = D.n_roots;
        D.d_max = b->dmax[g];
        D.m = b->m[g];
        D.slot = qi;
        D.pad = 0;
        if (i == 0 || items[i].key != items[i - 1].key) {
            Group G;
            G.cfg.ec = std::get<0>(items[i].key);
            G.cfg.subwarp = std::get<1>(items[i].key);
            G.cfg.chunk = std::get<2>(items[i].key);
            G.first = i;
            G.count = 0;
            G.d_cap = 0;
            G.k_max = 0;
            P.groups.push_back(G);
        }
        Group& G = P.groups.back();
        G.count++;
        if (D.k >= 3 && D.k <= D.d_max + 1) {
            G.d_cap = std::max(G.d_cap, D.d_max);
            G.k_max = std::max(G.k_max, D.k);
        }
    }
    for (Group& G : P.groups) {
        // item indices of a launch are 32-bit, and once the work runs out every
        // warp and block still advances the claim cursors by one chunk: below
        // 2^31 roots the cursors cannot wrap (the server's launches use the same bound)
        unsigned long long items = 0;
        for (uint32_t i = G.first; i < G.first + G.count; ++i) items += P.q[i].n_roots;
        if (items >= (1ull << 31))
            return set_error(KC_E_UNSUPPORTED, "one launch would hold %llu roots (at most 2^31 - 1)", items);
        if (G.k_max >= 3 && !batch_smem_bytes(G.d_cap, G.k_max, G.cfg))
            return set_error(KC_E_UNSUPPORTED, "a graph's out-degree %u is too large for a batched launch", G.d_cap);
        G.ws_off = off_ws;
        off_ws += al(batch_ws_bytes(G.count));
    }
    P.ws_bytes = off_ws;
    return KC_OK;
}

// descriptors to the device, then one launch sequence per group
static kc_status enqueue_plan(const kc_batch* b, const Plan& P, void* stage, char* ws, kc_result* results_dev,
                              cudaStream_t s) {
    if (P.q.empty()) return KC_OK;
    memcpy(stage, P.q.data(), P.q.size() * sizeof(QDesc));
    KC_CUDA(cudaMemcpyAsync(ws, stage, P.q.size() * sizeof(QDesc), cudaMemcpyHostToDevice, s));
    const QDesc* qd = (const QDesc*)ws;
    for (const Group& G : P.groups)
        KC_CHECK(batch_launch(qd + G.first, G.count, G.d_cap, G.k_max, G.cfg, ws + G.ws_off, b->g->time_limit_s,
                              b->g->sm_count, results_dev, nullptr, nullptr, s));
    return KC_OK;
}

static kc_status ensure_stage(kc_batch* b, size_t bytes) {
    if (b->staged_pending) {
        KC_CUDA(cudaEventSynchronize(b->staged));  // the previous call's copy has left the buffer
        b->staged_pending = false;
    }
    if (b->stage && b->stage_bytes >= bytes) return KC_OK;
    if (b->stage) cudaFreeHost(b->stage);
    b->stage = nullptr;
    b->stage_bytes = 0;
    KC_CUDA(cudaMallocHost(&b->stage, bytes));
    b->stage_bytes = bytes;
    return KC_OK;
}

}  // namespace kc

using namespace kc;

extern "C" {

kc_status kc_batch_create(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t nnz,
                          const uint32_t* graph_offsets, uint32_t num_graphs, int ptrs_on_device, int orient,
                          int validate, void* stream, kc_batch** out) {
    clear_error();
    if (!out) return set_error(KC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!graph_offsets) return set_error(KC_E_INVALID_ARG, "graph_offsets is NULL");
    if (num_graphs == 0) return set_error(KC_E_INVALID_ARG, "num_graphs must be >= 1");
    if (graph_offsets[0] != 0 || graph_offsets[num_graphs] != n)
        return set_error(KC_E_INVALID_ARG, "graph_offsets must start at 0 and end at n");
    for (uint32_t g = 0; g < num_graphs; ++g)
        if (graph_offsets[g + 1] < graph_offsets[g])
            return set_error(KC_E_INVALID_ARG, "graph_offsets must be non-decreasing");
    cudaStream_t s = (cudaStream_t)stream;
    kc_batch* b = new (std::nothrow) kc_batch();
    if (!b) return set_error(KC_E_NO_MEMORY, "host allocation failed");
    b->ng = num_graphs;
    b->off.assign(graph_offsets, graph_offsets + num_graphs + 1);
    DevBuf d_off, tmp;
    auto fail = [&](kc_status st) {
        dev_free(d_off);
        dev_free(tmp);
        kc_batch_destroy(b);
        return st;
    };
    kc_status st = dev_alloc(d_off, ((size_t)num_graphs + 1) * 4);
    if (st != KC_OK) return fail(st);
    cudaError_t e = cudaMemcpyAsync(d_off.ptr, graph_offsets, ((size_t)num_graphs + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(cuda_error(e, "copy graph offsets", __FILE__, __LINE__));
    if (validate && nnz) {
        // no edge may leave its graph's vertex range
        bool bad = false;
        if (!ptrs_on_device) {
            if (!row_ptr || !col_idx) return fail(set_error(KC_E_INVALID_ARG, "row_ptr or col_idx is NULL"));
            for (uint32_t g = 0; g < num_graphs && !bad; ++g)
                for (uint32_t v = graph_offsets[g]; v < graph_offsets[g + 1] && !bad; ++v)
                    for (uint64_t j = row_ptr[v]; j < row_ptr[v + 1] && j < nnz; ++j)
                        if (col_idx[j] < graph_offsets[g] || col_idx[j] >= graph_offsets[g + 1]) {
                            bad = true;
                            break;
                        }
        } else {
            st = dev_alloc(tmp, 16);
            if (st != KC_OK) return fail(st);
            unsigned flag = 0;
            e = cudaMemsetAsync(tmp.ptr, 0, 4, s);
            if (e == cudaSuccess) {
                k_check_blocks<<<std::max(1u, std::min(4096u, (n + 255) / 256)), 256, 0, s>>>(
                    row_ptr, col_idx, (const uint32_t*)d_off.ptr, num_graphs, n, (unsigned*)tmp.ptr);
                note_launch();
                e = cudaMemcpyAsync(&flag, tmp.ptr, 4, cudaMemcpyDeviceToHost, s);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(cuda_error(e, "graph block check", __FILE__, __LINE__));
            bad = flag != 0;
        }
        if (bad) return fail(set_error(KC_E_INVALID_GRAPH, "an edge joins two different graphs of the batch"));
    }
    st = kc_graph_create(row_ptr, col_idx, n, nnz, ptrs_on_device, orient, validate, stream, &b->g);
    if (st != KC_OK) {
        std::string msg = kc_last_error();
        dev_free(d_off);
        dev_free(tmp);
        kc_batch_destroy(b);
        return set_error(st, "%s", msg.c_str());
    }
    // roots grouped by graph (a stable pass over the union's out-degree order)
    st = dev_alloc(tmp, (size_t)n * 4 + 16);
    if (st == KC_OK) st = dev_alloc(b->roots, (size_t)n * 4 + 16);
    if (st != KC_OK) return fail(st);
    const unsigned nb = std::max(1u, std::min(4096u, (n + 255) / 256));
    if (n) {
        k_graph_of<<<nb, 256, 0, s>>>((const uint32_t*)b->g->old_of_new.ptr, (const uint32_t*)d_off.ptr, num_graphs, n,
                                      (uint32_t*)tmp.ptr);
        note_launch();
        st = sort_ids_by_key((const uint32_t*)tmp.ptr, n, num_graphs - 1, (uint32_t*)b->roots.ptr, b->g->tmp, s,
                             (const uint32_t*)b->g->roots.ptr);
        if (st != KC_OK) return fail(st);
    }
    DevBuf sizes;
    st = dev_alloc(sizes, (size_t)num_graphs * 12 + 16);
    if (st != KC_OK) return fail(st);
    unsigned long long* d_m = (unsigned long long*)sizes.ptr;
    uint32_t* d_dmax = (uint32_t*)(d_m + num_graphs);
    k_graph_sizes<<<num_graphs, 256, 0, s>>>((const uint32_t*)b->g->row_ptr.ptr, (const uint32_t*)b->roots.ptr,
                                             (const uint32_t*)d_off.ptr, d_m, d_dmax);
    note_launch();
    b->m.resize(num_graphs);
    b->dmax.resize(num_graphs);
    e = cudaMemcpyAsync(b->m.data(), d_m, (size_t)num_graphs * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dmax.data(), d_dmax, (size_t)num_graphs * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(sizes);
    if (e != cudaSuccess) return fail(cuda_error(e, "batch set-up", __FILE__, __LINE__));
    e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_error(e, "event", __FILE__, __LINE__));
    dev_free(d_off);
    dev_free(tmp);
    *out = b;
    return KC_OK;
}

kc_status kc_batch_destroy(kc_batch* b) {
    if (!b) return KC_OK;
    if (b->staged_pending) cudaEventSynchronize(b->staged);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->stage) cudaFreeHost(b->stage);
    dev_free(b->roots);
    dev_free(b->ws);
    if (b->g) kc_graph_destroy(b->g);
    delete b;
    return KC_OK;
}

kc_status kc_batch_graph_info(const kc_batch* b, uint32_t graph, uint32_t* n_out, uint64_t* m_out,
                              uint32_t* d_max_out) {
    clear_error();
    if (!b) return set_error(KC_E_INVALID_ARG, "NULL batch");
    if (graph >= b->ng) return set_error(KC_E_INVALID_ARG, "graph %u out of range", graph);
    if (n_out) *n_out = b->off[graph + 1] - b->off[graph];
    if (m_out) *m_out = b->m[graph];
    if (d_max_out) *d_max_out = b->dmax[graph];
    return KC_OK;
}

kc_status kc_batch_set_time_limit(kc_batch* b, double seconds) {
    clear_error();
    if (!b) return set_error(KC_E_INVALID_ARG, "NULL batch");
    return kc_graph_set_time_limit(b->g, seconds);
}

kc_status kc_batch_count(kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq,
                         kc_result* results_dev, const kc_tune* tune, void* stream) {
    clear_error();
    if (!b) return set_error(KC_E_INVALID_ARG, "NULL batch");
    if (nq == 0) return KC_OK;
    if (!graph_ids || !ks || !results_dev) return set_error(KC_E_INVALID_ARG, "NULL query or result array");
    cudaStream_t s = (cudaStream_t)stream;
    Plan P;
    KC_CHECK(make_plan(b, graph_ids, ks, nq, tune, nullptr, P));
    KC_CHECK(ensure_stage(b, P.q.size() * sizeof(QDesc) + 16));
    KC_CHECK(dev_alloc(b->ws, P.ws_bytes));
    KC_CHECK(enqueue_plan(b, P, b->stage, (char*)b->ws.ptr, results_dev, s));
    KC_CUDA(cudaEventRecord(b->staged, s));
    b->staged_pending = true;
    return KC_OK;
}

kc_status kc_batch_tune(kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq, uint32_t sample,
                        kc_tune* tune_out, void* stream) {
    clear_error();
    if (!b || !tune_out) return set_error(KC_E_INVALID_ARG, "NULL batch or tune_out");
    if (nq && (!graph_ids || !ks)) return set_error(KC_E_INVALID_ARG, "NULL query arrays");
    cudaStream_t s = (cudaStream_t)stream;
    if (sample == 0) sample = 256;
    // buckets (out-degree class, k) with their first `sample` queries
    std::map<std::pair<uint32_t, uint32_t>, std::vector<uint32_t>> buckets;
    for (uint32_t i = 0; i < nq; ++i) {
        if (graph_ids[i] >= b->ng) return set_error(KC_E_INVALID_ARG, "query %u: graph out of range", i);
        auto& v = buckets[{dclass_of(b->dmax[graph_ids[i]]), ks[i]}];
        if (v.size() < sample) v.push_back(i);
    }
    memset(tune_out, 0, sizeof(kc_tune));
    DevBuf res;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KC_CUDA(cudaEventCreate(&e0));
    KC_CUDA(cudaEventCreate(&e1));
    kc_status st = KC_OK;
    for (auto& kv : buckets) {
        const uint32_t dclass = kv.first.first, k = kv.first.second;
        if (tune_out->n >= KC_TUNE_MAX) break;
        std::vector<uint32_t> gid, kk;
        for (uint32_t i : kv.second) {
            gid.push_back(graph_ids[i]);
            kk.push_back(ks[i]);
        }
        const uint32_t m = (uint32_t)gid.size();
        std::vector<BatchConfig> cands;
        if (k < 3) {
            cands.push_back(prior_config(dclass, k));
        } else {
            for (int ec = 0; ec < 2; ++ec)
                for (uint32_t G : {2u, 4u, 8u, 32u})
                    for (uint32_t chunk : {4u, 32u}) {
                        if (dclass == 0 && (ec || G != 4)) continue;  // only small roots: groups unused
                        BatchConfig c;
                        c.ec = ec;
                        c.subwarp = G;
                        c.chunk = chunk;
                        cands.push_back(c);
                    }
        }
        float best = -1.f;
        BatchConfig bestc = prior_config(dclass, k);
        for (const BatchConfig& c : cands) {
            Plan P;
            st = make_plan(b, gid.data(), kk.data(), m, nullptr, &c, P);
            if (st != KC_OK) {
                clear_error();
                st = KC_OK;
                continue;  // does not fit this configuration
            }
            if ((st = ensure_stage(b, P.q.size() * sizeof(QDesc) + 16)) != KC_OK) break;
            if ((st = dev_alloc(b->ws, P.ws_bytes)) != KC_OK) break;
            if ((st = dev_alloc(res, (size_t)m * sizeof(kc_result) + 16)) != KC_OK) break;
            float ms = 0.f, t = 0.f;
            for (int rep = 0; rep < 2 && st == KC_OK; ++rep) {
                cudaEventRecord(e0, s);
                st = enqueue_plan(b, P, b->stage, (char*)b->ws.ptr, (kc_result*)res.ptr, s);
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) st = cuda_error(e, "tuning run", __FILE__, __LINE__);
                cudaEventElapsedTime(&t, e0, e1);
                ms = t;  // the second (warm) run is kept
            }
            if (st != KC_OK) break;
            if (best < 0.f || ms < best) {
                best = ms;
                bestc = c;
            }
        }
        if (st != KC_OK) break;
        kc_tune_entry& te = tune_out->e[tune_out->n++];
        te.dclass = dclass;
        te.k = k;
        te.scheme = bestc.ec ? KC_SCHEME_EC : KC_SCHEME_VC;
        te.subwarp = bestc.subwarp;
        te.chunk = bestc.chunk;
        te.ms = best < 0.f ? 0.f : best;
    }
    // The buckets were timed apart; together they share the launches and the
    // small-root cursor.  Time the assembled table on every query against
    // uniform configurations (one launch) and keep the fastest.
    if (st == KC_OK && nq) {
        std::vector<std::pair<bool, BatchConfig>> whole;
        whole.push_back({false, BatchConfig()});  // the table as tuned
        for (int ec = 0; ec < 2; ++ec)
            for (uint32_t G : {4u, 8u})
                for (uint32_t chunk : {4u, 32u, 128u}) {
                    BatchConfig c;
                    c.ec = ec;
                    c.subwarp = G;
                    c.chunk = chunk;
                    whole.push_back({true, c});
                }
        float best = -1.f;
        size_t besti = 0;
        for (size_t w = 0; w < whole.size() && st == KC_OK; ++w) {
            Plan P;
            kc_status ps = make_plan(b, graph_ids, ks, nq, tune_out, whole[w].first ? &whole[w].second : nullptr, P);
            if (ps != KC_OK) {
                clear_error();
                continue;
            }
            if ((st = ensure_stage(b, P.q.size() * sizeof(QDesc) + 16)) != KC_OK) break;
            if ((st = dev_alloc(b->ws, P.ws_bytes)) != KC_OK) break;
            if ((st = dev_alloc(res, (size_t)nq * sizeof(kc_result) + 16)) != KC_OK) break;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && st == KC_OK; ++rep) {
                cudaEventRecord(e0, s);
                st = enqueue_plan(b, P, b->stage, (char*)b->ws.ptr, (kc_result*)res.ptr, s);
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) st = cuda_error(e, "tuning run", __FILE__, __LINE__);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (st == KC_OK && (best < 0.f || ms < best)) {
                best = ms;
                besti = w;
            }
        }
        if (st == KC_OK && besti > 0)
            for (uint32_t i = 0; i < tune_out->n; ++i) {
                const BatchConfig& c = whole[besti].second;
                tune_out->e[i].scheme = c.ec ? KC_SCHEME_EC : KC_SCHEME_VC;
                tune_out->e[i].subwarp = c.subwarp;
                tune_out->e[i].chunk = c.chunk;
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(res);
    return st;
}

kc_status kc_batch_capture(kc_batch* b, const uint32_t* graph_ids, const uint32_t* ks, uint32_t nq,
                           kc_result* results_dev, const kc_tune* tune, kc_batch_exec** out) {
    clear_error();
    if (!b || !out) return set_error(KC_E_INVALID_ARG, "NULL batch or out");
    *out = nullptr;
    if (nq == 0) return set_error(KC_E_INVALID_ARG, "nq must be >= 1");
    if (!graph_ids || !ks || !results_dev) return set_error(KC_E_INVALID_ARG, "NULL query or result array");
    Plan P;
    KC_CHECK(make_plan(b, graph_ids, ks, nq, tune, nullptr, P));
    kc_batch_exec* x = new (std::nothrow) kc_batch_exec();
    if (!x) return set_error(KC_E_NO_MEMORY, "host allocation failed");
    auto fail = [&](kc_status st) {
        kc_batch_exec_destroy(x);
        return st;
    };
    kc_status st = dev_alloc(x->ws, P.ws_bytes);
    if (st != KC_OK) return fail(st);
    cudaError_t e = cudaMallocHost(&x->stage, P.q.size() * sizeof(QDesc) + 16);
    if (e != cudaSuccess) return fail(cuda_error(e, "staging", __FILE__, __LINE__));
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_error(e, "capture stream", __FILE__, __LINE__));
    cudaGraph_t graph = nullptr;
    const unsigned long long launches0 = kc_launch_count();
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        st = enqueue_plan(b, P, x->stage, (char*)x->ws.ptr, results_dev, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == KC_OK && e2 != cudaSuccess) st = cuda_error(e2, "end capture", __FILE__, __LINE__);
    } else {
        st = cuda_error(e, "begin capture", __FILE__, __LINE__);
    }
    if (st == KC_OK) {
        e = cudaGraphInstantiate(&x->exec, graph, 0);
        if (e != cudaSuccess) st = cuda_error(e, "graph instantiate", __FILE__, __LINE__);
    }
    x->kernels = kc_launch_count() - launches0;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != KC_OK) return fail(st);
    *out = x;
    return KC_OK;
}

kc_status kc_batch_exec_launch(kc_batch_exec* x, void* stream) {
    clear_error();
    if (!x || !x->exec) return set_error(KC_E_INVALID_ARG, "NULL executable");
    KC_CUDA(cudaGraphLaunch(x->exec, (cudaStream_t)stream));
    for (unsigned long long i = 0; i < x->kernels; ++i) note_launch();
    return KC_OK;
}

kc_status kc_batch_exec_destroy(kc_batch_exec* x) {
    if (!x) return KC_OK;
    if (x->exec) cudaGraphExecDestroy(x->exec);
    if (x->stage) cudaFreeHost(x->stage);
    dev_free(x->ws);
    delete x;
    return KC_OK;
}

}  // extern "C"
