// Serving loop (include/kclique.h, kc_server_*): a pool of resident oriented
// graphs and a worker thread that admits count queries as they arrive.
//
// With KC_SERVER_AUTO_TRAVERSAL and a time limit, adding a graph measures its
// cost profile (profile_graph): which (k, traversal) shapes finish within the
// limit on a slot's share of the SMs, and in how long.  A query takes the
// traversal its profile says finishes, and KC_SERVER_REFUSE_EXPENSIVE
// answers a shape that does not at once (KC_E_REFUSED).
//
// Orientation queries (pivot = 0) that the profile measured at most BATCH_MS
// (or that have no profile) and whose graphs fit the batched kernel wait in
// one queue; whenever a slot (a stream with its own working memory) is free,
// the worker packs up to max_batch of them, their profiled times adding up to
// at most half the time limit, into one persistent launch (batch_launch), so
// queries that arrive while others run start on the next free slot and their
// launches overlap on the device.  Each query's result is published to
// host-mapped memory by the thread that completes its last root, so it is
// served before the rest of its launch ends.  Pivot queries, longer
// orientation queries, and orientation queries whose bitmaps need global
// memory take a slot each and run through the graph's own path
// (kc_count_async), at most one per graph at a time (they share the graph's
// working memory).  Persistent launches hold their SMs until done, so every
// slot launches on a fixed share of the SMs (SMs / slots) and a long launch
// cannot starve the others.  A graph is admitted while the server's resident
// bytes stay within its device-memory budget, and a graph-path query while
// the device reports enough free memory for that path's buffers.  Waiting
// queries are admitted cheapest first (by a size estimate), except that a
// query waiting longer than a second goes before any cheaper one; the serial
// baseline keeps arrival order.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kc_common.cuh"

namespace kc {
namespace srv {

using Clock = std::chrono::steady_clock;

struct Ticket {
    uint32_t graph = 0, k = 0;
    int pivot = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    kc_result r{};
    int state = 0;  // 0 queued, 1 running, 2 done
    uint32_t launch = 0;
};

struct BatchSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    DevBuf ws;                    // descriptors, then every group's working memory
    DevBuf res;                   // final results of the launch
    kc_result* res_h = nullptr;   // pinned copy of res
    kc_result* early_h = nullptr; // mapped: results published early
    unsigned* done_h = nullptr;   // mapped: 1 once early_h[i] is written
    kc_result* early_d = nullptr;
    unsigned* done_d = nullptr;
    QDesc* stage = nullptr;       // pinned descriptors
    std::vector<uint64_t> tickets;
    std::vector<char> finished;
    bool busy = false;
    bool single = false;          // running one query through its graph's own path
    uint32_t graph = 0;           // that query's graph
};

static constexpr uint32_t MAX_GROUPS = 16;

static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t batch_slot_bytes(uint32_t cap) {
    return al((size_t)cap * sizeof(QDesc)) + MAX_GROUPS * al(batch_ws_bytes(cap));
}

}  // namespace srv
}  // namespace kc

using namespace kc;
using namespace kc::srv;

struct kc_server {
    int device = 0;
    int sms = 0;
    int share = 0;        // SMs' worth of blocks per launch: every slot's launch fits side by side
    size_t budget = 0;
    size_t resident = 0;
    uint32_t max_batch = 1;
    int flags = 0;
    double time_limit = 0;
    std::vector<kc_graph*> graphs;
    std::deque<Ticket> tickets;
    std::deque<uint64_t> q_batch, q_single;
    std::vector<BatchSlot> bs;
    std::vector<char> graph_busy;  // a single-path query of this graph is in flight
    // per graph, per (k, traversal) (shape_index): SHAPE_UNKNOWN, SHAPE_FITS
    // (finished within the time limit when the graph was profiled, in
    // shape_ms) or SHAPE_EXPENSIVE (ran out of it: at profiling, or a query
    // of that shape did; KC_SERVER_REFUSE_EXPENSIVE refuses the next ones)
    std::vector<std::vector<uint8_t>> shape_state;
    std::vector<std::vector<float>> shape_ms;
    std::vector<char> profiled;
    uint64_t refused = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    Clock::time_point t0;
    uint64_t launches = 0, served = 0;
    cudaStream_t setup = nullptr;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// Launch configuration of a query (the paper's guideline, Section 4.5).
BatchConfig config_of(uint32_t d_max, uint32_t k) {
    BatchConfig c;
    c.ec = k >= 6;
    c.subwarp = ((d_max + 31) / 32) <= 8 ? 4 : 8;
    c.chunk = 16;
    return c;
}

bool batchable(const kc_graph* g, uint32_t k, int pivot) {
    if (pivot) return false;
    if (k < 3 || k > g->d_max + 1) return true;
    if (k > 68) return false;
    return batch_smem_bytes(g->d_max, k, config_of(g->d_max, k)) != 0;
}

static constexpr uint32_t SHAPE_KMAX = 128;
static constexpr uint8_t SHAPE_UNKNOWN = 0, SHAPE_FITS = 1, SHAPE_EXPENSIVE = 2;
// the cost profile measures the orientation traversal up to this k
static constexpr uint32_t PROFILE_KMAX = 16;
// profiled orientation queries longer than this skip the batched kernel
static constexpr double BATCH_MS = 2.0;

size_t shape_index(uint32_t k, int pivot) { return (size_t)std::min<uint32_t>(k, SHAPE_KMAX - 1) * 2 + (pivot ? 1 : 0); }

void finish(kc_server* S, uint64_t t, const kc_result& r) {
    Ticket& T = S->tickets[t];
    T.r = r;
    T.t_done = S->now_ms();
    T.state = 2;
    S->served++;
    if (r.status == KC_E_TIMEOUT) S->shape_state[T.graph][shape_index(T.k, T.pivot)] = SHAPE_EXPENSIVE;
}

kc_result error_result(kc_status st) {
    kc_result r{};
    r.status = st;
    return r;
}

// Estimated cost of a queued query (cheapest first within admission).
double cost_of(const kc_server* S, uint64_t t) {
    const Ticket& T = S->tickets[t];
    const kc_graph* g = S->graphs[T.graph];
    return query_cost_estimate(g->m, g->d_max, T.k);
}

// Queries that waited this long are admitted before cheaper ones.
static constexpr double AGE_LIMIT_MS = 1000.0;

// Move the n cheapest queries of q (any that waited beyond AGE_LIMIT_MS
// first, oldest first) into out, in queue order.
void take_cheapest(kc_server* S, std::deque<uint64_t>& q, uint32_t n, std::vector<uint64_t>& out) {
    out.clear();
    if (S->flags & KC_SERVER_SERIAL) {  // the plain baseline keeps arrival order
        out.assign(q.begin(), q.begin() + std::min<size_t>(n, q.size()));
        q.erase(q.begin(), q.begin() + out.size());
        return;
    }
    if (n >= q.size()) {
        out.assign(q.begin(), q.end());
        q.clear();
        return;
    }
    const double now = S->now_ms();
    std::vector<std::pair<double, size_t>> key(q.size());
    for (size_t i = 0; i < q.size(); ++i) {
        const bool old = now - S->tickets[q[i]].t_submit > AGE_LIMIT_MS;
        key[i] = {old ? -1.0 - (double)(q.size() - i) : cost_of(S, q[i]), i};
    }
    std::nth_element(key.begin(), key.begin() + n, key.end());
    std::vector<char> pick(q.size(), 0);
    for (uint32_t j = 0; j < n; ++j) pick[key[j].second] = 1;
    std::deque<uint64_t> rest;
    for (size_t i = 0; i < q.size(); ++i) (pick[i] ? out.push_back(q[i]) : rest.push_back(q[i]));
    q.swap(rest);
}

// Pack up to max_batch queued orientation queries into one launch on slot b.
void launch_batch(kc_server* S, BatchSlot& b) {
    take_cheapest(S, S->q_batch, (uint32_t)std::min<size_t>(S->q_batch.size(), S->max_batch), b.tickets);
    // item indices of a launch are 32-bit: queries beyond 2^31 roots wait for the next launch
    // and one launch shares one deadline: its queries' profiled times add up
    // to at most half the time limit (queries without a profile count 0)
    unsigned long long roots = 0;
    double cost_ms = 0;
    const double budget_ms = S->time_limit > 0 ? 0.5e3 * S->time_limit : 0;
    size_t keep = 0;
    while (keep < b.tickets.size()) {
        const Ticket& T = S->tickets[b.tickets[keep]];
        const unsigned long long r = S->graphs[T.graph]->n;
        if (keep > 0 && roots + r >= (1ull << 31)) break;
        const size_t si = shape_index(T.k, 0);
        const double c = S->shape_state[T.graph][si] == SHAPE_FITS ? S->shape_ms[T.graph][si] : 0.0;
        if (keep > 0 && budget_ms > 0 && cost_ms + c > budget_ms) break;
        roots += r;
        cost_ms += c;
        ++keep;
    }
    for (size_t i = b.tickets.size(); i-- > keep;) S->q_batch.push_front(b.tickets[i]);
    b.tickets.resize(keep);
    const uint32_t n = (uint32_t)b.tickets.size();
    b.finished.assign(n, 0);
    // descriptors grouped by configuration
    struct Item {
        BatchConfig c;
        double cost;
        uint32_t i;
    };
    std::vector<Item> items(n);
    for (uint32_t i = 0; i < n; ++i) {
        const Ticket& T = S->tickets[b.tickets[i]];
        const kc_graph* g = S->graphs[T.graph];
        items[i].c = config_of(g->d_max, T.k);
        items[i].cost = query_cost_estimate(g->m, g->d_max, T.k);
        items[i].i = i;
    }
    auto key = [](const BatchConfig& c) { return (c.ec << 20) | (c.subwarp << 8) | c.chunk; };
    // one launch per configuration; inside one, cheapest queries first
    std::stable_sort(items.begin(), items.end(), [&](const Item& x, const Item& y) {
        return key(x.c) != key(y.c) ? key(x.c) < key(y.c) : x.cost < y.cost;
    });
    struct Grp {
        BatchConfig c;
        uint32_t first, count, d_cap, k_max;
    };
    std::vector<Grp> groups;
    for (uint32_t j = 0; j < n; ++j) {
        const Ticket& T = S->tickets[b.tickets[items[j].i]];
        const kc_graph* g = S->graphs[T.graph];
        QDesc& D = b.stage[j];
        D.rp = (const uint32_t*)g->row_ptr.ptr;
        D.col = (const uint32_t*)g->col.ptr;
        D.roots = (const uint32_t*)g->roots.ptr;
        D.n_roots = g->n;
        D.k = T.k;
        D.n = g->n;
        D.d_max = g->d_max;
        D.m = g->m;
        D.slot = items[j].i;
        D.pad = 0;
        // config_of yields at most four configurations (<= MAX_GROUPS)
        if (groups.empty() || key(groups.back().c) != key(items[j].c)) groups.push_back({items[j].c, j, 0, 0, 0});
        Grp& G = groups.back();
        G.count++;
        if (T.k >= 3 && T.k <= g->d_max + 1) {
            G.d_cap = std::max(G.d_cap, g->d_max);
            G.k_max = std::max(G.k_max, T.k);
        }
    }
    const uint32_t used = n;
    const double now = S->now_ms();
    const uint32_t launch = (uint32_t)++S->launches;
    for (uint32_t j = 0; j < used; ++j) {
        Ticket& T = S->tickets[b.tickets[items[j].i]];
        T.state = 1;
        T.t_admit = now;
        T.launch = launch;
    }
    memset(b.done_h, 0, (size_t)S->max_batch * 4);
    kc_status st = KC_OK;
    cudaError_t e = cudaMemcpyAsync(b.ws.ptr, b.stage, (size_t)used * sizeof(QDesc), cudaMemcpyHostToDevice, b.st);
    if (e != cudaSuccess) st = cuda_error(e, "descriptors", __FILE__, __LINE__);
    const QDesc* qd = (const QDesc*)b.ws.ptr;
    char* ws = (char*)b.ws.ptr + al((size_t)S->max_batch * sizeof(QDesc));
    for (size_t gi = 0; gi < groups.size() && st == KC_OK; ++gi) {
        const Grp& G = groups[gi];
        st = batch_launch(qd + G.first, G.count, G.d_cap, G.k_max, G.c, ws + gi * al(batch_ws_bytes(S->max_batch)),
                          S->time_limit, S->share, (kc_result*)b.res.ptr, b.early_d, b.done_d, b.st);
    }
    if (st == KC_OK) {
        e = cudaMemcpyAsync(b.res_h, b.res.ptr, (size_t)n * sizeof(kc_result), cudaMemcpyDeviceToHost, b.st);
        if (e == cudaSuccess) e = cudaEventRecord(b.ev, b.st);
        if (e != cudaSuccess) st = cuda_error(e, "batch results", __FILE__, __LINE__);
    }
    if (st != KC_OK) {
        cudaStreamSynchronize(b.st);
        for (uint32_t j = 0; j < used; ++j) finish(S, b.tickets[items[j].i], error_result(st));
        b.tickets.clear();
        return;
    }
    b.busy = true;  // result slot i <-> b.tickets[i]
}

// Run the queued single-path query at position pos of q_single on slot b.
void launch_single(kc_server* S, BatchSlot& b, size_t pos) {
    const uint64_t t = S->q_single[pos];
    S->q_single.erase(S->q_single.begin() + pos);
    Ticket& T = S->tickets[t];
    kc_graph* g = S->graphs[T.graph];
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    if (fr < ((size_t)256 << 20)) {  // too little free device memory for the pivot path's buffers
        finish(S, t, error_result(KC_E_NO_MEMORY));
        return;
    }
    T.state = 1;
    T.t_admit = S->now_ms();
    T.launch = (uint32_t)++S->launches;
    kc_status st = kc_count_async(g, T.k, T.pivot, KC_SCHEME_AUTO, 0, (kc_result*)b.res.ptr, nullptr, b.st);
    if (st == KC_OK) {
        cudaError_t e = cudaMemcpyAsync(b.res_h, b.res.ptr, sizeof(kc_result), cudaMemcpyDeviceToHost, b.st);
        if (e == cudaSuccess) e = cudaEventRecord(b.ev, b.st);
        if (e != cudaSuccess) st = cuda_error(e, "single result", __FILE__, __LINE__);
    }
    if (st != KC_OK) {
        cudaStreamSynchronize(b.st);
        finish(S, t, error_result(st));
        return;
    }
    b.tickets.assign(1, t);
    b.finished.assign(1, 0);
    b.single = true;
    b.graph = T.graph;
    S->graph_busy[T.graph] = 1;
    b.busy = true;
}

// The first queued single-path query (within a short look-ahead) whose
// graph has no single-path query in flight, or -1.
long next_single(kc_server* S) {
    if (S->flags & KC_SERVER_SERIAL) return S->q_single.empty() ? -1 : 0;
    const size_t look = std::min<size_t>(S->q_single.size(), 1024);
    const double now = S->now_ms();
    long best = -1;
    double best_cost = 0;
    for (size_t i = 0; i < look; ++i) {
        const uint64_t t = S->q_single[i];
        if (S->graph_busy[S->tickets[t].graph]) continue;
        if (now - S->tickets[t].t_submit > AGE_LIMIT_MS) return (long)i;  // waited too long: oldest first
        const double c = cost_of(S, t);
        if (best < 0 || c < best_cost) {
            best = (long)i;
            best_cost = c;
        }
    }
    return best;
}

void worker_main(kc_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    const bool serial = (S->flags & KC_SERVER_SERIAL) != 0;
    while (!S->stop) {
        bool progress = false, busy = false;
        for (BatchSlot& b : S->bs) {
            if (!b.busy) continue;
            if (!b.single)
                for (size_t i = 0; i < b.tickets.size(); ++i)
                    if (!b.finished[i] && *(volatile unsigned*)&b.done_h[i]) {
                        kc_result r;
                        memcpy(&r, (const void*)&b.early_h[i], sizeof(r));
                        finish(S, b.tickets[i], r);
                        b.finished[i] = 1;
                        progress = true;
                    }
            if (cudaEventQuery(b.ev) == cudaSuccess) {
                for (size_t i = 0; i < b.tickets.size(); ++i)
                    if (!b.finished[i]) finish(S, b.tickets[i], b.res_h[i]);
                if (b.single) S->graph_busy[b.graph] = 0;
                b.busy = false;
                b.single = false;
                progress = true;
            } else {
                busy = true;
            }
        }
        if (progress) S->cv_done.notify_all();
        // admission: every free slot takes the oldest waiting work it can run
        for (BatchSlot& b : S->bs) {
            if (b.busy) continue;
            if (serial && busy) break;
            const long si = next_single(S);
            const bool have_single = si >= 0;
            if (!have_single && S->q_batch.empty()) break;
            if (have_single && (S->q_batch.empty() || S->q_single[(size_t)si] < S->q_batch.front() ||
                                (!serial && cost_of(S, S->q_single[(size_t)si]) <= cost_of(S, S->q_batch.front()))))
                launch_single(S, b, (size_t)si);
            else
                launch_batch(S, b);
            progress = true;
            busy = busy || b.busy;
            if (serial) break;
        }
        if (progress) continue;
        if (busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

// Cost profile of a graph, measured when it is added (KC_SERVER_AUTO_TRAVERSAL
// with a time limit), on the SM share a query gets while serving: the
// orientation traversal at k = 3, 4, ... up to PROFILE_KMAX (and d_max + 1),
// each under the time limit, until one runs out of it (every larger k is
// then taken as expensive too: the search tree of k contains that of k - 1
// up to the size pruning).  If one ran out, the pivot traversal over every
// k (an upper bound of each fixed-k pivot count) and, should that run out as
// well, the pivot traversal at that k and up, until one runs out (the
// larger k are then expensive by pivoting too).  Nothing of the counts is
// kept.
void profile_graph(kc_graph* g, uint32_t d_max, std::vector<uint8_t>& st, std::vector<float>& ms, cudaStream_t s) {
    auto timed = [&](uint32_t k, int pivot, double& t_ms) {
        uint64_t total = 0;
        uint32_t flags = 0;
        const auto t0 = Clock::now();
        kc_status r = kc_count(g, k, pivot, KC_SCHEME_AUTO, 0, &total, nullptr, &flags, s);
        t_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        return r == KC_E_OVERFLOW ? KC_OK : r;
    };
    const uint32_t kmax = std::min<uint32_t>(d_max + 1, PROFILE_KMAX);
    uint32_t k_out = 0;
    for (uint32_t k = 3; k <= kmax; ++k) {
        double t = 0;
        const kc_status r = timed(k, 0, t);
        if (r == KC_OK) {
            st[shape_index(k, 0)] = SHAPE_FITS;
            ms[shape_index(k, 0)] = (float)t;
        } else {
            if (r == KC_E_TIMEOUT) {
                k_out = k;
                for (uint32_t j = k; j < SHAPE_KMAX; ++j) st[shape_index(j, 0)] = SHAPE_EXPENSIVE;
            }
            break;
        }
    }
    if (k_out == 0) return;
    std::vector<uint64_t> counts(SHAPE_KMAX);
    std::vector<uint8_t> ovf(SHAPE_KMAX);
    uint32_t omega = 0;
    const auto t0 = Clock::now();
    const kc_status r = kc_count_all(g, counts.data(), ovf.data(), SHAPE_KMAX, &omega, 0, nullptr, s);
    const double t = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    if (r == KC_OK || r == KC_E_OVERFLOW) {
        for (uint32_t j = 1; j < SHAPE_KMAX; ++j) {
            st[shape_index(j, 1)] = SHAPE_FITS;
            ms[shape_index(j, 1)] = (float)t;
        }
        return;
    }
    if (r != KC_E_TIMEOUT) return;
    for (uint32_t k = k_out; k <= kmax; ++k) {
        double t = 0;
        const kc_status rk = timed(k, 1, t);
        if (rk == KC_OK) {
            st[shape_index(k, 1)] = SHAPE_FITS;
            ms[shape_index(k, 1)] = (float)t;
        } else {
            if (rk == KC_E_TIMEOUT)
                for (uint32_t j = k; j < SHAPE_KMAX; ++j) st[shape_index(j, 1)] = SHAPE_EXPENSIVE;
            break;
        }
    }
}

// Traversal of a query: orientation unless the profile found it expensive,
// then pivoting unless that was found expensive too (then orientation).
// A graph without a profile follows the paper's guideline (Section 4.5):
// pivoting pays from k = 7 on.  The count is the same either way.
int auto_traversal(const kc_server* S, uint32_t graph_id, uint32_t k) {
    if (!S->profiled[graph_id]) return k >= 7 ? 1 : 0;
    const std::vector<uint8_t>& st = S->shape_state[graph_id];
    if (st[shape_index(k, 0)] != SHAPE_EXPENSIVE) return 0;
    return st[shape_index(k, 1)] != SHAPE_EXPENSIVE ? 1 : 0;
}

void free_slot(BatchSlot& b) {
    if (b.st) cudaStreamSynchronize(b.st);
    if (b.ev) cudaEventDestroy(b.ev);
    if (b.st) cudaStreamDestroy(b.st);
    dev_free(b.ws);
    dev_free(b.res);
    if (b.res_h) cudaFreeHost(b.res_h);
    if (b.early_h) cudaFreeHost(b.early_h);
    if (b.done_h) cudaFreeHost(b.done_h);
    if (b.stage) cudaFreeHost(b.stage);
}

}  // namespace

extern "C" {

kc_status kc_server_create(size_t hbm_budget, uint32_t max_batch, uint32_t slots, int flags, kc_server** out) {
    clear_error();
    if (!out) return set_error(KC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch == 0 || slots == 0) return set_error(KC_E_INVALID_ARG, "max_batch and slots must be >= 1");
    if (flags & ~(KC_SERVER_SERIAL | KC_SERVER_AUTO_TRAVERSAL | KC_SERVER_REFUSE_EXPENSIVE))
        return set_error(KC_E_INVALID_ARG, "unknown flags %d", flags);
    kc_server* S = new (std::nothrow) kc_server();
    if (!S) return set_error(KC_E_NO_MEMORY, "host allocation failed");
    S->flags = flags;
    S->max_batch = (flags & KC_SERVER_SERIAL) ? 1 : max_batch;
    if (flags & KC_SERVER_SERIAL) slots = 1;
    S->budget = hbm_budget;
    S->t0 = Clock::now();
    cudaGetDevice(&S->device);
    S->sms = sm_count_of_current_device();
    // persistent launches keep their SMs until their work is done, so each
    // slot gets a fixed share (all of it when serial)
    S->share = (flags & KC_SERVER_SERIAL) ? S->sms : std::max(1, S->sms / (int)slots);
    auto fail = [&](kc_status st) {
        kc_server_destroy(S);
        return st;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&S->setup, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_error(e, "stream", __FILE__, __LINE__));
    S->bs.resize(slots);
    for (BatchSlot& b : S->bs) {
        e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&b.res_h, (size_t)S->max_batch * sizeof(kc_result), 0);
        if (e == cudaSuccess)
            e = cudaHostAlloc((void**)&b.early_h, (size_t)S->max_batch * sizeof(kc_result), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&b.done_h, (size_t)S->max_batch * 4, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&b.stage, (size_t)S->max_batch * sizeof(QDesc), 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&b.early_d, b.early_h, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&b.done_d, b.done_h, 0);
        if (e != cudaSuccess) return fail(cuda_error(e, "batch slot", __FILE__, __LINE__));
        kc_status st = dev_alloc(b.ws, batch_slot_bytes(S->max_batch));
        if (st == KC_OK && b.res_h == nullptr) st = set_error(KC_E_NO_MEMORY, "host allocation failed");
        if (st == KC_OK) st = dev_alloc(b.res, (size_t)S->max_batch * sizeof(kc_result));
        if (st != KC_OK) return fail(st);
        S->resident += b.ws.bytes + b.res.bytes;
    }
    if (S->resident > S->budget)
        return fail(set_error(KC_E_NO_MEMORY, "the slots alone (%zu bytes) exceed the budget", S->resident));
    S->worker = std::thread(worker_main, S);
    *out = S;
    return KC_OK;
}

kc_status kc_server_add_graph(kc_server* S, const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n,
                              uint64_t nnz, int ptrs_on_device, int orient, int validate, uint32_t* graph_id) {
    clear_error();
    if (!S || !graph_id) return set_error(KC_E_INVALID_ARG, "NULL server or graph_id");
    kc_graph* g = nullptr;
    KC_CHECK(kc_graph_create(row_ptr, col_idx, n, nnz, ptrs_on_device, orient, validate, S->setup, &g));
    kc_graph_info info;
    kc_graph_info_get(g, &info);
    double limit = 0;
    int share = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        limit = S->time_limit;
        share = S->share;
    }
    std::vector<uint8_t> st(2 * SHAPE_KMAX, SHAPE_UNKNOWN);
    std::vector<float> ms(2 * SHAPE_KMAX, 0.0f);
    const bool profile = (S->flags & KC_SERVER_AUTO_TRAVERSAL) && limit > 0;
    if (profile) {
        // outside the lock: the worker keeps serving meanwhile
        kc_graph_set_time_limit(g, limit);
        g->sm_count = share;
        profile_graph(g, info.d_max, st, ms, S->setup);
        clear_error();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->resident + info.device_bytes > S->budget) {
        kc_graph_destroy(g);
        return set_error(KC_E_NO_MEMORY, "graph of %llu bytes exceeds the server budget",
                         (unsigned long long)info.device_bytes);
    }
    kc_graph_set_time_limit(g, S->time_limit);
    g->sm_count = S->share;  // launches of the graph path take one share too
    S->resident += info.device_bytes;
    *graph_id = (uint32_t)S->graphs.size();
    S->graphs.push_back(g);
    S->graph_busy.push_back(0);
    S->shape_state.push_back(std::move(st));
    S->shape_ms.push_back(std::move(ms));
    S->profiled.push_back(profile ? 1 : 0);
    return KC_OK;
}

kc_status kc_server_set_time_limit(kc_server* S, double seconds) {
    clear_error();
    if (!S) return set_error(KC_E_INVALID_ARG, "NULL server");
    if (!(seconds >= 0)) return set_error(KC_E_INVALID_ARG, "time limit must be >= 0");
    std::lock_guard<std::mutex> lk(S->mu);
    S->time_limit = seconds;
    for (kc_graph* g : S->graphs) kc_graph_set_time_limit(g, seconds);
    return KC_OK;
}

kc_status kc_server_submit(kc_server* S, uint32_t graph_id, uint32_t k, int pivot, uint64_t* ticket) {
    clear_error();
    if (!S || !ticket) return set_error(KC_E_INVALID_ARG, "NULL server or ticket");
    if (k == 0) return set_error(KC_E_INVALID_ARG, "k must be >= 1");
    if (pivot != 0 && pivot != 1) return set_error(KC_E_INVALID_ARG, "pivot must be 0 or 1");
    std::lock_guard<std::mutex> lk(S->mu);
    if (graph_id >= S->graphs.size()) return set_error(KC_E_INVALID_ARG, "unknown graph %u", graph_id);
    Ticket T;
    T.graph = graph_id;
    T.k = k;
    T.pivot = (S->flags & KC_SERVER_AUTO_TRAVERSAL) ? auto_traversal(S, graph_id, k) : pivot;
    T.t_submit = S->now_ms();
    const uint64_t id = S->tickets.size();
    S->tickets.push_back(T);
    *ticket = id;
    if ((S->flags & KC_SERVER_REFUSE_EXPENSIVE) &&
        S->shape_state[graph_id][shape_index(k, T.pivot)] == SHAPE_EXPENSIVE) {
        // this shape runs out of the time limit (profile or an earlier query): answer at once
        Ticket& R = S->tickets[id];
        R.r = error_result(KC_E_REFUSED);
        R.t_admit = R.t_done = R.t_submit;
        R.state = 2;
        S->refused++;
        S->cv_done.notify_all();
        return KC_OK;
    }
    pivot = T.pivot;
    // a query the profile measured above BATCH_MS runs through its graph's
    // own path (the single-graph kernels; one such query per graph at a time)
    const size_t si = shape_index(k, 0);
    const bool long_query = S->profiled[graph_id] && !pivot && S->shape_state[graph_id][si] == SHAPE_FITS &&
                            S->shape_ms[graph_id][si] > BATCH_MS;
    if (!long_query && batchable(S->graphs[graph_id], k, pivot))
        S->q_batch.push_back(id);
    else
        S->q_single.push_back(id);
    S->cv_work.notify_one();
    return KC_OK;
}

kc_status kc_server_poll(kc_server* S, uint64_t ticket, kc_server_result* out, int timeout_ms) {
    clear_error();
    if (!S || !out) return set_error(KC_E_INVALID_ARG, "NULL server or out");
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket >= S->tickets.size()) return set_error(KC_E_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    auto ready = [&] { return S->tickets[ticket].state == 2; };
    if (timeout_ms < 0)
        S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return set_error(KC_E_TIMEOUT, "ticket %llu not finished yet", (unsigned long long)ticket);
    const Ticket& T = S->tickets[ticket];
    out->total = T.r.total;
    out->total_hi = T.r.total_hi;
    out->flags = T.r.flags;
    out->status = T.r.status;
    out->graph_id = T.graph;
    out->k = T.k;
    out->pivot = T.pivot;
    out->launch = T.launch;
    out->t_submit_ms = T.t_submit;
    out->t_admit_ms = T.t_admit;
    out->t_done_ms = T.t_done;
    return KC_OK;
}

kc_status kc_server_stats(kc_server* S, uint64_t* launches, uint64_t* served, uint64_t* resident_bytes) {
    clear_error();
    if (!S) return set_error(KC_E_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (launches) *launches = S->launches;
    if (served) *served = S->served;
    if (resident_bytes) *resident_bytes = S->resident;
    return KC_OK;
}

kc_status kc_server_shape(kc_server* S, uint32_t graph_id, uint32_t k, int pivot, int* state, double* ms) {
    clear_error();
    if (!S || !state) return set_error(KC_E_INVALID_ARG, "NULL server or state");
    if (pivot != 0 && pivot != 1) return set_error(KC_E_INVALID_ARG, "pivot must be 0 or 1");
    std::lock_guard<std::mutex> lk(S->mu);
    if (graph_id >= S->graphs.size()) return set_error(KC_E_INVALID_ARG, "unknown graph %u", graph_id);
    const size_t i = shape_index(k, pivot);
    *state = S->shape_state[graph_id][i];
    if (ms) *ms = S->shape_ms[graph_id][i];
    return KC_OK;
}

kc_status kc_server_destroy(kc_server* S) {
    if (!S) return KC_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (BatchSlot& b : S->bs) free_slot(b);
    for (kc_graph* g : S->graphs) kc_graph_destroy(g);
    if (S->setup) cudaStreamDestroy(S->setup);
    delete S;
    return KC_OK;
}

}  // extern "C"
