// Orientation traversal (Fig. 2) without the binary encoding: the
// comparison point of Section 3.4 and of the ablation in Section 4.3
// (Fig. 6).  A candidate set is a sorted list of vertex ids, and
// I' = I ∩ N+(u) is computed by searching every member of I in the DAG row
// of u (binary search over the sorted row), which is how traversals that do
// not extract a binary-encoded induced sub-graph intersect.  One warp per
// work item: a root vertex (vertex-centric) or a root edge (edge-centric,
// Section 3.2).  The work units are the membership tests; they are also
// added per SM, for the load-balance measurement of Fig. 7.  The same walk
// lists the cliques (the listing the paper's conclusion names as a use of
// the traversal): in its EMIT form every member of a last intersection is
// written out with the vertices on its path.
#include <algorithm>
#include <cstring>

#include "kc_common.cuh"
#include "kc_dfs.cuh"

namespace kc {

static constexpr int LBLOCK = 256;
static constexpr int LWARPS = LBLOCK / 32;

struct ListParams {
    const uint32_t* rp;             // DAG row pointers (library numbering)
    const uint32_t* col;            // DAG columns, rows ascending
    uint32_t k;                     // 3 <= k <= LIST_MAX_K
    uint32_t n;                     // vertices
    const uint32_t* roots;          // VC: vertices in decreasing out-degree
    uint32_t n_items;               // VC: roots with out-degree >= k - 1; EC: DAG edges
    int ec;
    uint32_t dcap;                  // entries per stack level (the largest out-degree)
    uint32_t* lists;                // per warp: max(k - 3, 1) levels of dcap entries
    unsigned* cursor;               // next unclaimed item (zeroed before the launch)
    unsigned long long* sm_work;    // nullable: work units per SM (SM_WORK_SLOTS entries)
    Ctl* ctl;
    // listing (the EMIT kernel only): clique i goes to out[i k .. i k + k)
    // in the input numbering, for i < cap; emitted counts every clique found
    uint32_t* out;
    unsigned long long cap;
    unsigned long long* emitted;
    const uint32_t* old_of_new;
};

// Source vertex of DAG edge e: the largest v with rp[v] <= e (one thread).
__device__ __forceinline__ uint32_t edge_source(const uint32_t* __restrict__ rp, uint32_t n, uint32_t e) {
    uint32_t lo = 0, hi = n;  // rp[lo] <= e < rp[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(rp + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Whether x is in the sorted row col[b, e) (one thread).
__device__ __forceinline__ bool row_has(const uint32_t* __restrict__ col, uint32_t b, uint32_t e, uint32_t x) {
    while (b < e) {
        const uint32_t mid = (b + e) >> 1;
        const uint32_t y = __ldg(col + mid);
        if (y == x) return true;
        if (y < x) b = mid + 1; else e = mid;
    }
    return false;
}

// The members of L[from, to) that are out-neighbours of u, by the 32 lanes
// (each searches its members in N+(u)).  Writes them in order to out when
// out is not null; returns their number (the same in every lane).
__device__ __forceinline__ uint32_t list_intersect(const uint32_t* L, uint32_t from, uint32_t to,
                                                   const uint32_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                   uint32_t u, uint32_t* out, int lane) {
    const uint32_t b = __ldg(rp + u), e = __ldg(rp + u + 1);
    uint32_t cnt = 0;
    for (uint32_t base = from; base < to; base += 32) {
        const uint32_t i = base + (uint32_t)lane;
        bool hit = false;
        uint32_t x = 0;
        if (i < to) {
            x = L[i];
            hit = row_has(col, b, e, x);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (out && hit) out[cnt + __popc(bal & lanemask_lt())] = x;
        cnt += __popc(bal);
    }
    return cnt;
}

// Listing form of the last intersection: every member x of L[from, to)
// that is an out-neighbour of u closes the clique path + {x} (path: plen
// vertices, the same in every lane).  The warp reserves the slots of each
// 32 members with one atomic; a clique whose slot is at or beyond P.cap is
// counted but not written.  Returns the number of cliques closed.
__device__ uint32_t list_emit(const ListParams& P, const uint32_t* L, uint32_t from, uint32_t to, uint32_t u,
                              const uint32_t* path, uint32_t plen, int lane) {
    const uint32_t b = __ldg(P.rp + u), e = __ldg(P.rp + u + 1);
    uint32_t cnt = 0;
    for (uint32_t base = from; base < to; base += 32) {
        const uint32_t i = base + (uint32_t)lane;
        bool hit = false;
        uint32_t x = 0;
        if (i < to) {
            x = L[i];
            hit = row_has(P.col, b, e, x);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (bal == 0) continue;
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(P.emitted, (unsigned long long)__popc(bal));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (hit) {
            const unsigned long long slot = first + (unsigned long long)__popc(bal & lanemask_lt());
            if (slot < P.cap) {
                uint32_t* o = P.out + slot * P.k;
                for (uint32_t t = 0; t < plen; ++t) o[t] = __ldg(P.old_of_new + path[t]);
                o[plen] = __ldg(P.old_of_new + x);
            }
        }
        cnt += __popc(bal);
    }
    return cnt;
}

// One work item by one warp: the subtree of root v below its level-0
// candidates j_first .. j_end - 1 (VC: all of N+(v); EC: the one root edge
// v -> N+(v)[j_first]).  Levels are sorted lists: level 0 is v's DAG row,
// level l + 1 the members of level l after the chosen vertex u that are
// out-neighbours of u.  With two vertices left to choose, the members of
// the intersection are counted instead of stored.  stk: this warp's lists,
// (k - 3) levels of dcap entries.  Counts go to acc (the same in every
// lane), membership tests to work; stop is set when the time limit passed.
template <bool EMIT>
__device__ void list_walk(const ListParams& P, uint32_t v, uint32_t j_first, uint32_t j_end, uint32_t* stk,
                          Acc& acc, unsigned long long& work, int lane, bool& stop) {
    const uint32_t b0 = __ldg(P.rp + v);
    const uint32_t d = __ldg(P.rp + v + 1) - b0;
    const uint32_t* Lv[LIST_MAX_K];
    uint32_t S[LIST_MAX_K], J[LIST_MAX_K], E[LIST_MAX_K];
    const uint32_t R0 = P.k - 1;  // vertices still to choose at level 0, the chosen one included
    int l = 0;
    Lv[0] = P.col + b0;
    S[0] = d;
    J[0] = j_first;
    E[0] = min(j_end, d);
    uint32_t steps = 0;
    for (;;) {
        const uint32_t R = R0 - (uint32_t)l;
        if (J[l] >= E[l] || S[l] - J[l] < R) {  // no candidate left, or too few for R more vertices
            if (l == 0) break;
            --l;
            continue;
        }
        if ((++steps & 63u) == 0) {
            const int to = lane == 0 ? (int)timed_out(P.ctl) : 0;
            if (__shfl_sync(0xffffffffu, to, 0)) {
                stop = true;
                break;
            }
        }
        const uint32_t* L = Lv[l];
        const uint32_t u = L[J[l]];
        const uint32_t from = J[l] + 1, to = S[l];
        J[l] = from;
        work += to - from;
        if (R == 2) {  // u and one more: every common member closes a clique
            if (EMIT) {
                // the clique's other vertices: the root and the vertex chosen at
                // each level (the one just before that level's cursor)
                uint32_t path[LIST_MAX_K];
                path[0] = v;
                for (int t = 0; t <= l; ++t) path[1 + t] = Lv[t][J[t] - 1];
                acc.add(list_emit(P, L, from, to, u, path, (uint32_t)l + 2, lane));
            } else {
                acc.add(list_intersect(L, from, to, P.rp, P.col, u, nullptr, lane));
            }
            continue;
        }
        uint32_t* out = stk + (size_t)l * P.dcap;
        const uint32_t cnt = list_intersect(L, from, to, P.rp, P.col, u, out, lane);
        __syncwarp();  // the list is read by every lane below
        if (cnt < R - 1) continue;
        ++l;
        Lv[l] = out;
        S[l] = cnt;
        J[l] = 0;
        E[l] = cnt;
    }
}

// Persistent warps claim work items from a global cursor: roots (VC, in
// decreasing out-degree) or DAG edges (EC).
template <bool EMIT>
__global__ void __launch_bounds__(LBLOCK) k_count_list(const ListParams P) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = blockIdx.x * LWARPS + (threadIdx.x >> 5);
    const uint32_t nl = P.k > 3 ? P.k - 3 : 1;
    uint32_t* stk = P.lists + (size_t)gw * nl * P.dcap;
    Acc acc;
    unsigned long long work = 0;
    bool stop = false;
    while (!stop) {
        uint32_t i = 0;
        if (lane == 0) i = timed_out(P.ctl) ? NONE : atomicAdd(P.cursor, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i == NONE || i >= P.n_items) break;
        uint32_t v, j0, j1;
        if (P.ec) {
            uint32_t src = 0;
            if (lane == 0) src = edge_source(P.rp, P.n, i);
            v = __shfl_sync(0xffffffffu, src, 0);
            j0 = i - __ldg(P.rp + v);
            j1 = j0 + 1;
        } else {
            v = P.roots[i];
            j0 = 0;
            j1 = NONE;
        }
        list_walk<EMIT>(P, v, j0, j1, stk, acc, work, lane, stop);
    }
    // every lane holds the same totals: lane 0 publishes them
    if (lane == 0) {
        add_u128(&P.ctl->total_lo, &P.ctl->total_hi, acc.lo);
        if (acc.hi) atomicAdd(&P.ctl->total_hi, acc.hi);
        atomicAdd(&P.ctl->words, work);
        if (P.sm_work) {
            const unsigned sm = smid();
            if (sm < SM_WORK_SLOTS) atomicAdd(&P.sm_work[sm], work);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static kc_status list_geometry(const kc_graph* g, uint32_t k, int* blocks, size_t* words) {
    int bps = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_count_list<true>, LBLOCK, 0));
    if (bps < 1) return set_error(KC_E_UNSUPPORTED, "list traversal kernel cannot be resident");
    *blocks = bps * g->sm_count;
    const size_t nl = k > 3 ? k - 3 : 1;
    *words = (size_t)(*blocks) * LWARPS * nl * std::max<uint32_t>(g->d_max, 1);
    return KC_OK;
}

size_t list_scratch_words(const kc_graph* g, uint32_t k) {
    int blocks = 0;
    size_t words = 0;
    if (k < 3 || k > LIST_MAX_K || list_geometry(g, k, &blocks, &words) != KC_OK) return 0;
    return words;
}

kc_status list_launch(kc_graph* g, uint32_t k, bool ec, Ctl* ctl, unsigned* cursor, unsigned long long* sm_work,
                      cudaStream_t s, uint32_t* out, unsigned long long cap, unsigned long long* emitted) {
    if (k < 3 || k > LIST_MAX_K)
        return set_error(KC_E_UNSUPPORTED, "the list traversal takes 3 <= k <= %u", LIST_MAX_K);
    int blocks = 0;
    size_t words = 0;
    KC_CHECK(list_geometry(g, k, &blocks, &words));
    uint64_t n_items = 0;
    if (ec) {
        n_items = g->m;
    } else {
        for (uint64_t d = k - 1; d < g->outdeg_hist.size(); ++d) n_items += g->outdeg_hist[d];
    }
    // the claim cursor overshoots by one per warp once the items run out
    if (n_items + (uint64_t)blocks * LWARPS >= (1ull << 32))
        return set_error(KC_E_UNSUPPORTED, "%llu work items exceed the list traversal's 32-bit cursor",
                         (unsigned long long)n_items);
    if (n_items == 0) return KC_OK;
    KC_CHECK(dev_alloc(g->scratch, (words + 64) * 4));
    ListParams P;
    memset(&P, 0, sizeof(P));
    P.rp = (const uint32_t*)g->row_ptr.ptr;
    P.col = (const uint32_t*)g->col.ptr;
    P.k = k;
    P.n = g->n;
    P.roots = (const uint32_t*)g->roots.ptr;
    P.n_items = (uint32_t)n_items;
    P.ec = ec ? 1 : 0;
    P.dcap = std::max<uint32_t>(g->d_max, 1);
    P.lists = (uint32_t*)g->scratch.ptr;
    P.cursor = cursor;
    P.sm_work = sm_work;
    P.ctl = ctl;
    if (emitted) {
        P.out = out;
        P.cap = out ? cap : 0ull;
        P.emitted = emitted;
        P.old_of_new = (const uint32_t*)g->old_of_new.ptr;
        k_count_list<true><<<blocks, LBLOCK, 0, s>>>(P);
    } else {
        k_count_list<false><<<blocks, LBLOCK, 0, s>>>(P);
    }
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

}  // namespace kc
