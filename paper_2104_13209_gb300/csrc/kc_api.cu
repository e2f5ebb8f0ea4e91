// The public C ABI of libkclique (include/kclique.h): handles, argument
// checks, error messages, host<->device marshalling and dispatch to the
// orientation and counting kernels.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>

#include <mutex>

#include "kc_common.cuh"

namespace kc {

static thread_local std::string t_err;
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

kc_status set_error(kc_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

void clear_error() { t_err.clear(); }

kc_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    cudaGetLastError();  // a non-sticky error must not leak into the next call
    if (e == cudaErrorMemoryAllocation)
        return set_error(KC_E_NO_MEMORY, "out of device memory in %s (%s:%d)", what, file, line);
    return set_error(KC_E_CUDA, "CUDA error %d (%s) in %s (%s:%d)", (int)e, cudaGetErrorString(e), what, file, line);
}

kc_status dev_alloc(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.ptr && b.bytes >= bytes) return KC_OK;
    if (b.ptr) {
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        return set_error(KC_E_NO_MEMORY, "cudaMalloc of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return KC_OK;
}

void dev_free(DevBuf& b) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

static cudaMemPool_t scratch_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = 1ull << 30;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

kc_status scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    cudaMemPool_t pool = scratch_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s) : cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(KC_E_NO_MEMORY, "device scratch of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    }
    return KC_OK;
}

void scratch_free(void* p, cudaStream_t s) {
    if (!p) return;
    if (cudaFreeAsync(p, s) != cudaSuccess) cudaGetLastError();
}

static bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace kc

uint64_t kc_graph::device_bytes() const {
    const kc::DevBuf* bufs[] = {&row_ptr, &col, &new_of_old, &old_of_new, &core, &roots, &ctl,
                                &result, &pivot_out, &pv_stage, &scratch, &pv, &tmp, &sm_work};
    uint64_t t = 0;
    for (auto* b : bufs) t += b->bytes;
    return t;
}

using namespace kc;

extern "C" {

const char* kc_last_error(void) { return t_err.c_str(); }

const char* kc_status_name(kc_status s) {
    switch (s) {
        case KC_OK: return "KC_OK";
        case KC_E_INVALID_ARG: return "KC_E_INVALID_ARG";
        case KC_E_INVALID_GRAPH: return "KC_E_INVALID_GRAPH";
        case KC_E_NO_MEMORY: return "KC_E_NO_MEMORY";
        case KC_E_OVERFLOW: return "KC_E_OVERFLOW";
        case KC_E_TIMEOUT: return "KC_E_TIMEOUT";
        case KC_E_CUDA: return "KC_E_CUDA";
        case KC_E_INTERNAL: return "KC_E_INTERNAL";
        case KC_E_UNSUPPORTED: return "KC_E_UNSUPPORTED";
        case KC_E_REFUSED: return "KC_E_REFUSED";
        default: return "KC_E_UNKNOWN";
    }
}

int kc_version(void) { return KC_VERSION; }

uint64_t kc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

kc_status kc_graph_create(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t nnz,
                          int ptrs_on_device, int orient, int validate, void* stream, kc_graph** out) {
    clear_error();
    if (!out) return set_error(KC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!row_ptr) return set_error(KC_E_INVALID_ARG, "row_ptr is NULL");
    if (nnz > 0 && !col_idx) return set_error(KC_E_INVALID_ARG, "col_idx is NULL with nnz > 0");
    if (nnz >= (1ull << 32)) return set_error(KC_E_UNSUPPORTED, "nnz must be below 2^32");
    if (n == 0xFFFFFFFFu) return set_error(KC_E_UNSUPPORTED, "n must be below 2^32 - 1");
    if (orient != KC_ORIENT_DEGREE && orient != KC_ORIENT_DEGENERACY)
        return set_error(KC_E_INVALID_ARG, "unknown orientation %d", orient);
    if (nnz % 2) return set_error(KC_E_INVALID_GRAPH, "nnz is odd, so the CSR cannot be symmetric");
    cudaStream_t s = (cudaStream_t)stream;
    kc_graph* g = new (std::nothrow) kc_graph();
    if (!g) return set_error(KC_E_NO_MEMORY, "host allocation failed");
    cudaGetDevice(&g->device);
    g->sm_count = sm_count_of_current_device();
    g->n = n;
    g->m = nnz / 2;
    g->orient = orient;
    DevBuf in_rp, in_ci;
    const uint32_t* d_rp = row_ptr;
    const uint32_t* d_ci = col_idx;
    kc_status st = KC_OK;
    if (!ptrs_on_device) {
        if (!validate) {
            if (row_ptr[0] != 0 || row_ptr[n] != nnz) st = set_error(KC_E_INVALID_GRAPH, "row_ptr[0] or row_ptr[n] wrong");
        }
        if (st == KC_OK) st = dev_alloc(in_rp, ((size_t)n + 1) * 4);
        if (st == KC_OK) st = dev_alloc(in_ci, (size_t)nnz * 4 + 4);
        if (st == KC_OK) {
            cudaError_t e = cudaMemcpyAsync(in_rp.ptr, row_ptr, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && nnz)
                e = cudaMemcpyAsync(in_ci.ptr, col_idx, (size_t)nnz * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) st = cuda_error(e, "copy CSR to device", __FILE__, __LINE__);
        }
        d_rp = (const uint32_t*)in_rp.ptr;
        d_ci = (const uint32_t*)in_ci.ptr;
    }
    if (st == KC_OK && nnz == 0) {
        if (!in_ci.ptr) st = dev_alloc(in_ci, 16);
        if (st == KC_OK && !d_ci) d_ci = (const uint32_t*)in_ci.ptr;
    }
    if (st == KC_OK) st = build_graph(g, d_rp, d_ci, validate, s);
    if (st == KC_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "graph build", __FILE__, __LINE__);
    }
    dev_free(in_rp);
    dev_free(in_ci);
    if (st != KC_OK) {
        kc_graph_destroy(g);
        return st;
    }
    *out = g;
    return KC_OK;
}

kc_status kc_graph_destroy(kc_graph* g) {
    if (!g) return KC_OK;
    DevBuf* bufs[] = {&g->row_ptr, &g->col, &g->new_of_old, &g->old_of_new, &g->core, &g->roots, &g->ctl,
                       &g->result, &g->pivot_out, &g->pv_stage, &g->scratch, &g->pv, &g->tmp, &g->sm_work};
    for (auto* b : bufs) dev_free(*b);
    delete g;
    return KC_OK;
}

kc_status kc_graph_info_get(const kc_graph* g, kc_graph_info* out) {
    clear_error();
    if (!g || !out) return set_error(KC_E_INVALID_ARG, "NULL argument");
    out->n = g->n;
    out->d_max = g->d_max;
    out->num_edges = g->m;
    out->degeneracy = g->degeneracy;
    out->orient = g->orient;
    out->device_bytes = g->device_bytes();
    out->orient_ms = g->orient_ms;
    return KC_OK;
}

kc_status kc_graph_set_time_limit(kc_graph* g, double seconds) {
    clear_error();
    if (!g) return set_error(KC_E_INVALID_ARG, "NULL graph");
    if (!(seconds >= 0.0)) return set_error(KC_E_INVALID_ARG, "time limit must be >= 0");
    g->time_limit_s = seconds;
    return KC_OK;
}

kc_status kc_graph_last_work(const kc_graph* g, uint64_t* units) {
    clear_error();
    if (!g || !units) return set_error(KC_E_INVALID_ARG, "NULL argument");
    *units = g->last_work;
    return KC_OK;
}

kc_status kc_graph_last_sm_work(const kc_graph* g, uint64_t* per_sm, uint32_t cap, uint32_t* slots_out) {
    clear_error();
    if (!g || !slots_out) return set_error(KC_E_INVALID_ARG, "NULL argument");
    if (cap && !per_sm) return set_error(KC_E_INVALID_ARG, "per_sm is NULL");
    std::vector<uint64_t> w(SM_WORK_SLOTS, 0);
    if (g->sm_work.ptr) KC_CUDA(cudaMemcpy(w.data(), g->sm_work.ptr, SM_WORK_SLOTS * 8, cudaMemcpyDeviceToHost));
    uint32_t slots = (uint32_t)std::max(g->sm_count, 0);
    for (uint32_t i = 0; i < SM_WORK_SLOTS; ++i)
        if (w[i]) slots = std::max(slots, i + 1);
    for (uint32_t i = 0; i < cap; ++i) per_sm[i] = i < SM_WORK_SLOTS ? w[i] : 0;
    *slots_out = slots;
    return KC_OK;
}

kc_status kc_graph_export(const kc_graph* g, uint32_t* dag_row_ptr, uint32_t* dag_col, uint32_t* new_of_old,
                          uint32_t* core) {
    clear_error();
    if (!g) return set_error(KC_E_INVALID_ARG, "NULL graph");
    if (dag_row_ptr) KC_CUDA(cudaMemcpy(dag_row_ptr, g->row_ptr.ptr, ((size_t)g->n + 1) * 4, cudaMemcpyDeviceToHost));
    if (dag_col && g->m) KC_CUDA(cudaMemcpy(dag_col, g->col.ptr, (size_t)g->m * 4, cudaMemcpyDeviceToHost));
    if (new_of_old && g->n) KC_CUDA(cudaMemcpy(new_of_old, g->new_of_old.ptr, (size_t)g->n * 4, cudaMemcpyDeviceToHost));
    if (core) {
        if (g->orient != KC_ORIENT_DEGENERACY) return set_error(KC_E_INVALID_ARG, "core numbers need degeneracy orientation");
        if (g->n) KC_CUDA(cudaMemcpy(core, g->core.ptr, (size_t)g->n * 4, cudaMemcpyDeviceToHost));
    }
    return KC_OK;
}

// whether orientation-mode per-vertex counts of size k run in the
// orientation traversal (else the pivoting one serves them)
static bool orient_per_vertex(const kc_graph* g, uint32_t k) {
    return k >= 3 && (uint64_t)k <= (uint64_t)g->d_max + 1 && deep_supported(g, k, true);
}

static kc_status resolve(const kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, CountArgs& a) {
    if (!g) return set_error(KC_E_INVALID_ARG, "NULL graph");
    if (k == 0) return set_error(KC_E_INVALID_ARG, "k must be >= 1");
    if (pivot != 0 && pivot != 1) return set_error(KC_E_INVALID_ARG, "pivot must be 0 or 1");
    if (scheme != KC_SCHEME_AUTO && scheme != KC_SCHEME_VC && scheme != KC_SCHEME_EC && scheme != KC_SCHEME_VC_LIST &&
        scheme != KC_SCHEME_EC_LIST)
        return set_error(KC_E_INVALID_ARG, "unknown scheme %d", scheme);
    if (subwarp != 0 && subwarp != 1 && subwarp != 2 && subwarp != 4 && subwarp != 8 && subwarp != 16 && subwarp != 32)
        return set_error(KC_E_INVALID_ARG, "subwarp must be 0, 1, 2, 4, 8, 16 or 32");
    a.k = k;
    a.pivot = pivot;
    // Section 4.5: vertex-centric for k < 6, edge-centric from k = 6 on
    a.scheme = scheme == KC_SCHEME_AUTO ? (k < 6 ? KC_SCHEME_VC : KC_SCHEME_EC) : scheme;
    if (a.scheme == KC_SCHEME_EC && k < 3) a.scheme = KC_SCHEME_VC;
    if (subwarp == 0) {
        // Section 4.5: few threads per group for small out-degrees, 8 for large
        uint32_t W = (g->d_max + 31) / 32;
        subwarp = W <= 8 ? 4 : 8;
    }
    a.subwarp = subwarp;
    a.per_vertex_dev = nullptr;
    return KC_OK;
}

static bool list_scheme(int scheme) { return scheme == KC_SCHEME_VC_LIST || scheme == KC_SCHEME_EC_LIST; }

kc_status kc_count_async(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, kc_result* result_dev,
                         uint64_t* per_vertex_dev, void* stream) {
    clear_error();
    CountArgs a;
    KC_CHECK(resolve(g, k, pivot, scheme, subwarp, a));
    if (!result_dev) return set_error(KC_E_INVALID_ARG, "result_dev is NULL");
    if (per_vertex_dev && !is_device_pointer(per_vertex_dev))
        return set_error(KC_E_INVALID_ARG, "per_vertex_dev must be device memory");
    if (!pivot && per_vertex_dev && list_scheme(a.scheme))
        return set_error(KC_E_UNSUPPORTED, "the list traversal gives totals only");
    // per-vertex counts: from the traversal the call names, except for
    // k <= 2 (closed forms in the pivoting path) and sizes the orientation
    // traversal does not take
    if (pivot || (per_vertex_dev && !orient_per_vertex(g, k)))
        return count_pivot_async(g, k, result_dev, per_vertex_dev, (cudaStream_t)stream);
    a.per_vertex_dev = per_vertex_dev;
    return count_launch(g, a, result_dev, (cudaStream_t)stream);
}

kc_status kc_graph_reserve(kc_graph* g, uint32_t k_max, int pivot, int per_vertex, void* stream) {
    clear_error();
    if (!g) return set_error(KC_E_INVALID_ARG, "NULL graph");
    return count_reserve(g, k_max, pivot, per_vertex, (cudaStream_t)stream);
}

static kc_status count_sync(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, uint64_t* lo_out,
                            uint64_t* hi_out, uint64_t* per_vertex_out, uint32_t* flags_out, void* stream) {
    if (!lo_out) return set_error(KC_E_INVALID_ARG, "total_out is NULL");
    CountArgs a;
    KC_CHECK(resolve(g, k, pivot, scheme, subwarp, a));
    if (!pivot && per_vertex_out && list_scheme(a.scheme))
        return set_error(KC_E_UNSUPPORTED, "the list traversal gives totals only");
    // per-vertex counts: as in kc_count_async
    if (per_vertex_out && !orient_per_vertex(g, k)) pivot = 1;
    cudaStream_t s = (cudaStream_t)stream;
    KC_CHECK(dev_alloc(g->result, sizeof(kc_result) + 64));
    kc_result* rd = (kc_result*)g->result.ptr;
    uint64_t* pv_dev = nullptr;
    const bool pv_host = per_vertex_out && !is_device_pointer(per_vertex_out);
    if (per_vertex_out) {
        if (pv_host) {
            KC_CHECK(dev_alloc(g->pv_stage, ((size_t)g->n + 1) * 8));
            pv_dev = (uint64_t*)g->pv_stage.ptr;
        } else {
            pv_dev = per_vertex_out;
        }
    }
    if (pivot) {
        KC_CHECK(count_pivot_async(g, k, rd, pv_dev, s));
    } else {
        a.per_vertex_dev = pv_dev;
        KC_CHECK(count_launch(g, a, rd, s));
    }
    kc_result r;
    KC_CUDA(cudaMemcpyAsync(&r, rd, sizeof(r), cudaMemcpyDeviceToHost, s));
    if (pv_host && g->n) KC_CUDA(cudaMemcpyAsync(per_vertex_out, pv_dev, (size_t)g->n * 8, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    g->last_work = r.words;
    *lo_out = r.total;
    if (hi_out) *hi_out = r.total_hi;
    if (flags_out) *flags_out = r.flags;
    if (r.status == KC_E_INTERNAL && g->ctl.ptr) {
        // the first failed device-side check, if one was recorded
        Ctl hc;
        KC_CUDA(cudaMemcpy(&hc, g->ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost));
        return set_error(KC_E_INTERNAL, "device reported KC_E_INTERNAL (check %u refused index %u)", hc.dbg_code,
                         hc.dbg_idx);
    }
    if (r.status != KC_OK) return set_error((kc_status)r.status, "device reported %s", kc_status_name(r.status));
    if (r.flags & (KC_FLAG_TOTAL_OVERFLOW | KC_FLAG_VERTEX_OVERFLOW))
        return set_error(KC_E_OVERFLOW, "a count exceeded 2^64 - 1");
    return KC_OK;
}

kc_status kc_count128(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, uint64_t* lo_out,
                      uint64_t* hi_out, uint32_t* flags_out, void* stream) {
    clear_error();
    return count_sync(g, k, pivot, scheme, subwarp, lo_out, hi_out, nullptr, flags_out, stream);
}

kc_status kc_count(kc_graph* g, uint32_t k, int pivot, int scheme, uint32_t subwarp, uint64_t* total_out,
                   uint64_t* per_vertex_out, uint32_t* flags_out, void* stream) {
    clear_error();
    uint64_t hi = 0;
    return count_sync(g, k, pivot, scheme, subwarp, total_out, &hi, per_vertex_out, flags_out, stream);
}

kc_status kc_list_cliques(kc_graph* g, uint32_t k, uint32_t* cliques_dev, uint64_t cap, uint64_t* count_out,
                          void* stream) {
    clear_error();
    if (!g || !count_out) return set_error(KC_E_INVALID_ARG, "NULL argument");
    if (k == 0) return set_error(KC_E_INVALID_ARG, "k must be >= 1");
    if (k < 3 || k > LIST_MAX_K) return set_error(KC_E_UNSUPPORTED, "listing takes 3 <= k <= %u", LIST_MAX_K);
    if (cap && !cliques_dev) return set_error(KC_E_INVALID_ARG, "cliques_dev is NULL");
    if (cap && !is_device_pointer(cliques_dev)) return set_error(KC_E_INVALID_ARG, "cliques_dev must be device memory");
    if (cap > UINT64_MAX / k) return set_error(KC_E_INVALID_ARG, "cap too large");
    cudaStream_t s = (cudaStream_t)stream;
    KC_CHECK(dev_alloc(g->result, sizeof(kc_result) + 64));
    kc_result* rd = (kc_result*)g->result.ptr;
    KC_CHECK(list_cliques_launch(g, k, cliques_dev, cap, rd, s));
    kc_result r;
    KC_CUDA(cudaMemcpyAsync(&r, rd, sizeof(r), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    g->last_work = r.words;
    *count_out = r.total;
    if (r.status != KC_OK) return set_error((kc_status)r.status, "device reported %s", kc_status_name(r.status));
    if (r.total_hi) return set_error(KC_E_OVERFLOW, "more than 2^64 - 1 cliques");
    return KC_OK;
}

static kc_status count_all_common(kc_graph* g, uint64_t* counts_lo, uint64_t* counts_hi, uint8_t* overflow64,
                                  uint8_t* overflow128, uint32_t cap, uint32_t* omega_out, uint32_t per_vertex_k,
                                  uint64_t* per_vertex_out, void* stream) {
    if (!g) return set_error(KC_E_INVALID_ARG, "NULL graph");
    if (!counts_lo) return set_error(KC_E_INVALID_ARG, "counts is NULL");
    if (cap == 0) return set_error(KC_E_INVALID_ARG, "cap must be >= 1");
    if (per_vertex_out && per_vertex_k == 0) return set_error(KC_E_INVALID_ARG, "per_vertex_k must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* pv_dev = nullptr;
    const bool pv_host = per_vertex_out && !is_device_pointer(per_vertex_out);
    if (per_vertex_out) {
        if (pv_host) {
            KC_CHECK(dev_alloc(g->pv_stage, ((size_t)g->n + 1) * 8));
            pv_dev = (uint64_t*)g->pv_stage.ptr;
        } else {
            pv_dev = per_vertex_out;
        }
    }
    std::vector<uint64_t> hi(cap);
    std::vector<uint8_t> o128(cap);
    uint32_t flags = 0, omega = 0;
    KC_CHECK(count_all_run(g, cap, per_vertex_out ? per_vertex_k : 0, pv_dev, counts_lo, hi.data(), o128.data(),
                           &omega, &flags, s));
    if (pv_host && g->n) {
        KC_CUDA(cudaMemcpyAsync(per_vertex_out, pv_dev, (size_t)g->n * 8, cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
    }
    if (counts_hi) memcpy(counts_hi, hi.data(), (size_t)cap * 8);
    bool any64 = (flags & KC_FLAG_VERTEX_OVERFLOW) != 0, any128 = false;
    for (uint32_t j = 0; j < cap; ++j) {
        const bool o64 = hi[j] != 0 || o128[j] != 0;
        if (overflow64) overflow64[j] = o64 ? 1 : 0;
        if (overflow128) overflow128[j] = o128[j];
        any64 |= o64;
        any128 |= o128[j] != 0;
    }
    if (omega_out) *omega_out = omega;
    if (flags & KC_FLAG_TIMEOUT) return set_error(KC_E_TIMEOUT, "time limit reached");
    if (flags & KC_FLAG_INTERNAL) return set_error(KC_E_INTERNAL, "device-side consistency check failed");
    if (counts_hi ? (any128 || (flags & KC_FLAG_VERTEX_OVERFLOW)) : any64)
        return set_error(KC_E_OVERFLOW, counts_hi ? "a count exceeded 2^128 - 1" : "a count exceeded 2^64 - 1");
    return KC_OK;
}

kc_status kc_count_all(kc_graph* g, uint64_t* counts, uint8_t* overflow, uint32_t cap, uint32_t* omega_out,
                       uint32_t per_vertex_k, uint64_t* per_vertex_out, void* stream) {
    clear_error();
    return count_all_common(g, counts, nullptr, overflow, nullptr, cap, omega_out, per_vertex_k, per_vertex_out,
                            stream);
}

kc_status kc_count_all128(kc_graph* g, uint64_t* counts_lo, uint64_t* counts_hi, uint8_t* overflow, uint32_t cap,
                          uint32_t* omega_out, uint32_t per_vertex_k, uint64_t* per_vertex_out, void* stream) {
    clear_error();
    if (!counts_hi) return set_error(KC_E_INVALID_ARG, "counts_hi is NULL");
    return count_all_common(g, counts_lo, counts_hi, nullptr, overflow, cap, omega_out, per_vertex_k,
                            per_vertex_out, stream);
}

}  // extern "C"
