// Graph-orientation k-clique counting (Fig. 2; Sections 2.4, 3.2-3.6).
//
// Work items are root vertices (vertex-centric, VC) or root DAG edges
// (edge-centric, EC).  For each item the candidate set C (VC: N+(r); EC:
// N+(u) ∩ N+(v)) is listed in ascending library id, and its induced sub-graph
// is binary-encoded (Section 3.4): row i has bit j set iff C[j] is an
// out-neighbour of C[i].  Because the library numbering is a topological
// order, every row only has bits j > i.
//
// The tree below the item is then walked depth-first with an explicit stack
// (Section 3.3).  At a tree node with candidate list I (a bitmap) and `rem`
// vertices still to choose:
//   rem == 1:  count += popc(I)
//   rem == 2:  count += sum over j in I of popc(I & row_j)      (two levels at once)
//   rem >= 3:  for each v in I (ascending): I' = I & row_v, descend with rem - 1,
//              skipping v when fewer than rem bits of I remain or
//              popc(I') < rem - 1 (no clique of the needed size can follow).
//
// Two execution modes share one persistent kernel:
//   block mode (|C| > 32): the whole block builds the bitmap in shared memory
//     (or per-block global scratch when it does not fit); groups of G threads
//     (G = 1..32, Section 3.5) take the level-below-root subtrees one at a
//     time from a shared counter and split every word-wise AND across their
//     threads;
//   warp mode (|C| <= 32): one warp per item, every row is one 32-bit word,
//     and every lane walks its own subtree.
// Items are taken from global counters (persistent blocks, Section 3.6); VC
// roots are ordered by decreasing out-degree so the largest trees start first.
// Counts are summed per thread, then per block, then into an exact 128-bit
// total with carry detection.
#include "kc_common.cuh"

namespace kc {

static constexpr int BLOCK = 256;
static constexpr int NWARPS = BLOCK / 32;
static constexpr int SMALL_D = 32;      // warp mode handles |C| <= 32
static constexpr int WARP_DEPTH = 32;   // per-lane stack levels in warp mode
static constexpr int MAX_DEPTH = 64;    // stack levels per group in block mode (k <= MAX_DEPTH + 4)
static constexpr uint32_t NONE = 0xFFFFFFFFu;

struct CountParams {
    const uint32_t* rp;        // DAG row pointers (library numbering)
    const uint32_t* col;       // DAG columns
    uint32_t n;
    uint32_t k;
    // work lists
    const uint32_t* big_items;    // block-mode items (VC: root ids; EC: DAG edge ids)
    const unsigned* big_count_dev;  // if non-null, number of big items is read here (EC deferred list)
    uint32_t big_count;
    const uint32_t* small_items;  // warp-mode items
    uint32_t small_count;
    uint32_t* defer_items;        // EC warp phase: items with |C| > 32 are appended here
    unsigned* defer_count;
    const uint32_t* edge_src;     // EC: source of each DAG edge
    // geometry
    uint32_t dcap;             // max |C| in block mode
    uint32_t wcap;             // words per bitmap row = ceil(dcap / 32)
    uint32_t depth;            // stack levels per group in block mode
    int bitmap_in_smem;
    int stack_in_smem;
    uint32_t* gscratch;        // per-block global scratch base
    size_t gscratch_words;     // words per block
    Ctl* ctl;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    const unsigned lane = threadIdx.x & 31;
    return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
}

template <int G>
__device__ __forceinline__ void group_sync(unsigned gm) {
    if (G > 1) __syncwarp(gm);
}

template <int G>
__device__ __forceinline__ uint32_t group_sum(uint32_t x, unsigned gm) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(gm, x, o);
    return x;
}

__device__ __forceinline__ void acc_add(unsigned long long& lo, unsigned long long& hi, unsigned long long x) {
    lo += x;
    hi += (lo < x) ? 1ull : 0ull;
}

// First set bit of L at position >= from, scanning words up to hi (inclusive).
__device__ __forceinline__ uint32_t next_bit(const uint32_t* L, uint32_t from, uint32_t hi) {
    uint32_t w = from >> 5;
    if (w > hi) return NONE;
    uint32_t bits = L[w] & (0xFFFFFFFFu << (from & 31));
    while (bits == 0) {
        if (++w > hi) return NONE;
        bits = L[w];
    }
    return (w << 5) + (__ffs(bits) - 1);
}

// binary search of x in sorted s[lo, hi); returns index or NONE
__device__ __forceinline__ uint32_t find_sorted(const uint32_t* s, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint32_t y = s[mid];
        if (y == x) return mid;
        if (y < x) lo = mid + 1; else hi = mid;
    }
    return NONE;
}

// ---------------------------------------------------------------------------
// Block mode
// ---------------------------------------------------------------------------
struct BlockShared {
    uint32_t item;
    uint32_t d;
    uint32_t root_u, root_v;
    uint32_t task_next;
    uint32_t scan_carry;
    uint32_t warp_tot[NWARPS];
};

// Candidate set into cand[]: VC copies N+(r); EC intersects N+(u), N+(v).
__device__ uint32_t block_load_candidates(const CountParams& P, bool ec, uint32_t u, uint32_t v, uint32_t* cand,
                                          BlockShared& sh) {
    const uint32_t* col = P.col;
    if (!ec) {
        uint32_t b = P.rp[u], d = P.rp[u + 1] - b;
        for (uint32_t i = threadIdx.x; i < d; i += BLOCK) cand[i] = col[b + i];
        return d;
    }
    // EC: walk the shorter list, binary-search each element in the longer one,
    // compact the hits in order with a block-wide scan per 256-element chunk.
    uint32_t bu = P.rp[u], du = P.rp[u + 1] - bu;
    uint32_t bv = P.rp[v], dv = P.rp[v + 1] - bv;
    const uint32_t* A = col + bu;  // searched
    const uint32_t* B = col + bv;  // walked
    uint32_t na = du, nb = dv;
    if (du < dv) { A = col + bv; na = dv; B = col + bu; nb = du; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) sh.scan_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += BLOCK) {
        uint32_t i = base + threadIdx.x;
        uint32_t x = 0;
        bool hit = false;
        if (i < nb) {
            x = B[i];
            hit = find_sorted(A, 0, na, x) != NONE;
        }
        unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) sh.warp_tot[warp] = __popc(bal);
        __syncthreads();
        uint32_t off = sh.scan_carry;
        for (int w2 = 0; w2 < warp; ++w2) off += sh.warp_tot[w2];
        if (hit) cand[off + __popc(bal & lanemask_lt())] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w2 = 0; w2 < NWARPS; ++w2) t += sh.warp_tot[w2];
            sh.scan_carry += t;
        }
        __syncthreads();
    }
    return sh.scan_carry;
}

// Rows of the induced sub-graph: bit j of row i iff cand[j] in N+(cand[i]).
// One warp per row; lanes take 32 consecutive entries of N+(cand[i]) at a
// time and binary-search them among cand[i+1 .. d).
__device__ void block_build_bitmap(const CountParams& P, const uint32_t* cand, uint32_t d, uint32_t W, uint32_t* bm) {
    for (uint32_t x = threadIdx.x; x < d * W; x += BLOCK) bm[x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t last = cand[d - 1];
    for (uint32_t i = warp; i < d; i += NWARPS) {
        const uint32_t x = cand[i];
        const uint32_t b = P.rp[x], e = P.rp[x + 1];
        uint32_t* row = bm + (size_t)i * W;
        for (uint32_t j0 = b; j0 < e; j0 += 32) {
            uint32_t j = j0 + lane;
            uint32_t y = j < e ? P.col[j] : NONE;
            if (y != NONE && y <= last) {
                uint32_t pos = find_sorted(cand, i + 1, d, y);
                if (pos != NONE) atomicOr(&row[pos >> 5], 1u << (pos & 31));
            }
            if (__shfl_sync(0xffffffffu, y, 31) >= last) break;  // the rest of the row is beyond cand
        }
    }
    __syncthreads();
}

// sum over j in I of popc(I & row_j), words [lo, hi]; thread gl of the group
// takes the words lo + gl, lo + gl + G, ...
template <int G>
__device__ __forceinline__ void edge_count(const uint32_t* I, const uint32_t* bm, uint32_t W, uint32_t lo, uint32_t hi,
                                           unsigned gl, unsigned long long& alo, unsigned long long& ahi) {
    for (uint32_t w = lo + gl; w <= hi; w += G) {
        uint32_t bits = I[w];
        while (bits) {
            uint32_t j = (w << 5) + (__ffs(bits) - 1);
            bits &= bits - 1;
            const uint32_t* rj = bm + (size_t)j * W;
            uint32_t s = 0;
            for (uint32_t x = w; x <= hi; ++x) s += __popc(I[x] & rj[x]);
            acc_add(alo, ahi, s);
        }
    }
}

template <int G>
__device__ void group_walk(const CountParams& P, const uint32_t* bm, uint32_t d, uint32_t W, uint32_t rem0,
                           uint32_t* stk, BlockShared& sh, unsigned long long& alo, unsigned long long& ahi) {
    const unsigned gm = group_mask<G>();
    const unsigned gl = threadIdx.x & (G - 1);
    const unsigned leader = (threadIdx.x & 31) & ~(unsigned)(G - 1);
    uint32_t cur[MAX_DEPTH + 2];
    uint32_t idx[MAX_DEPTH + 2];
    uint32_t cnt[MAX_DEPTH + 2];
    const uint32_t hiw = W - 1;
    for (;;) {
        uint32_t t = 0;
        if (gl == 0) t = atomicAdd(&sh.task_next, 1u);
        t = __shfl_sync(gm, t, leader);
        if (t >= d) break;
        const uint32_t* R = bm + (size_t)t * W;
        const uint32_t lo0 = (t + 1) >> 5;
        if (rem0 == 0) {
            if (gl == 0) acc_add(alo, ahi, 1);
            continue;
        }
        if (rem0 == 1) {
            uint32_t s = 0;
            for (uint32_t w = lo0 + gl; w <= hiw; w += G) s += __popc(R[w]);
            acc_add(alo, ahi, s);
            continue;
        }
        if (rem0 == 2) {
            edge_count<G>(R, bm, W, lo0, hiw, gl, alo, ahi);
            continue;
        }
        // rem0 >= 3: explicit-stack DFS; level 0 list is the bitmap row itself
        uint32_t c0 = 0;
        for (uint32_t w = lo0 + gl; w <= hiw; w += G) c0 += __popc(R[w]);
        c0 = group_sum<G>(c0, gm);
        if (c0 < rem0) continue;
        int l = 0;
        cur[0] = t;
        idx[0] = 0;
        cnt[0] = c0;
        for (;;) {
            const uint32_t* L = (l == 0) ? R : stk + (size_t)(l - 1) * W;
            const uint32_t rem = rem0 - l;
            uint32_t v = (cnt[l] - idx[l] < rem) ? NONE : next_bit(L, cur[l] + 1, hiw);
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
            group_sync<G>(gm);  // readers of C (previous sibling) are done
            uint32_t c = 0;
            for (uint32_t w = lo + gl; w <= hiw; w += G) {
                uint32_t x = L[w] & rv[w];
                C[w] = x;
                c += __popc(x);
            }
            c = group_sum<G>(c, gm);
            group_sync<G>(gm);
            const uint32_t need = rem - 1;
            if (c < need) continue;
            if (need == 2) {
                edge_count<G>(C, bm, W, lo, hiw, gl, alo, ahi);
                continue;
            }
            ++l;
            cur[l] = v;
            idx[l] = 0;
            cnt[l] = c;
        }
    }
}

template <int G, bool EC>
__device__ void block_phase(const CountParams& P, uint32_t* smem, BlockShared& sh, unsigned long long& alo,
                            unsigned long long& ahi) {
    const uint32_t W = P.wcap;
    uint32_t* cand = smem;
    uint32_t* bm;
    uint32_t* stk_base;
    uint32_t* gs = P.gscratch + (size_t)blockIdx.x * P.gscratch_words;
    uint32_t* sp = smem + ((P.dcap + 31) & ~31u);
    if (P.bitmap_in_smem) {
        bm = sp;
        sp += (size_t)P.dcap * W;
    } else {
        bm = gs;
        gs += (size_t)P.dcap * W;
    }
    if (P.stack_in_smem) stk_base = sp; else stk_base = gs;
    const uint32_t ngroups = BLOCK / G;
    uint32_t* stk = stk_base + (size_t)(threadIdx.x / G) * P.depth * W;
    (void)ngroups;
    const uint32_t s0 = EC ? 2 : 1;
    const uint32_t rem0 = P.k - s0 - 1;  // vertices to choose below a level-(s0+1) task
    const uint32_t nbig = P.big_count_dev ? *(volatile const unsigned*)P.big_count_dev : P.big_count;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t i = atomicAdd(&P.ctl->work_next, 1u);
            sh.item = i < nbig ? P.big_items[i] : NONE;
            sh.task_next = 0;
        }
        __syncthreads();
        const uint32_t item = sh.item;
        if (item == NONE) break;
        uint32_t u, v = 0;
        if (EC) {
            u = P.edge_src[item];
            v = P.col[item];
        } else {
            u = item;
        }
        uint32_t d = block_load_candidates(P, EC, u, v, cand, sh);
        __syncthreads();
        if (d + s0 >= P.k && d > 0) {
            const uint32_t Wd = (d + 31) >> 5;  // words per row for this item
            block_build_bitmap(P, cand, d, Wd, bm);
            group_walk<G>(P, bm, d, Wd, rem0, stk, sh, alo, ahi);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Warp mode (|C| <= 32): rows are single words
// ---------------------------------------------------------------------------
struct WarpShared {
    uint32_t cand[32];
    uint32_t row[32];
    uint32_t stk[WARP_DEPTH * 32];
};

// sum over j in c of popc(c & row_j)
__device__ __forceinline__ uint32_t edge_count1(uint32_t c, const uint32_t* row) {
    uint32_t s = 0;
    while (c) {
        uint32_t j = __ffs(c) - 1;
        c &= c - 1;
        s += __popc(c & row[j]);
    }
    return s;
}

// count of rem-subsets of J (ascending choice) that are cliques, with rem >= 3
__device__ uint64_t lane_walk(uint32_t J0, uint32_t rem0, const uint32_t* row, uint32_t* stk) {
    const int lane = threadIdx.x & 31;
    uint64_t acc = 0;
    int l = 0;
    stk[lane] = J0;
    for (;;) {
        uint32_t J = stk[l * 32 + lane];
        const uint32_t rem = rem0 - l;
        if ((uint32_t)__popc(J) < rem) {
            if (l == 0) break;
            --l;
            continue;
        }
        uint32_t v = __ffs(J) - 1;
        J &= J - 1;
        stk[l * 32 + lane] = J;
        uint32_t c = J & row[v];
        const uint32_t need = rem - 1;
        if ((uint32_t)__popc(c) < need) continue;
        if (need == 2) {
            acc += edge_count1(c, row);
            continue;
        }
        ++l;
        stk[l * 32 + lane] = c;
    }
    return acc;
}

template <bool EC>
__device__ void warp_phase(const CountParams& P, WarpShared& ws, unsigned long long& alo, unsigned long long& ahi) {
    const int lane = threadIdx.x & 31;
    const uint32_t s0 = EC ? 2 : 1;
    const uint32_t rem0 = P.k - s0 - 1;
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(&P.ctl->work_next_small, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= P.small_count) break;
        const uint32_t item = P.small_items[i];
        uint32_t d;
        if (!EC) {
            const uint32_t b = P.rp[item];
            d = P.rp[item + 1] - b;
            if (d + s0 < P.k) continue;  // cannot hold a k-clique
            if (lane < (int)d) ws.cand[lane] = P.col[b + lane];
        } else {
            const uint32_t u = P.edge_src[item], v = P.col[item];
            uint32_t bu = P.rp[u], du = P.rp[u + 1] - bu;
            uint32_t bv = P.rp[v], dv = P.rp[v + 1] - bv;
            if (du + 1 < P.k - 1 || dv + 1 < P.k - 1) continue;  // |C| <= min(du, dv) too small
            const uint32_t* A = P.col + bu;
            const uint32_t* B = P.col + bv;
            uint32_t na = du, nb = dv;
            if (du < dv) { A = P.col + bv; na = dv; B = P.col + bu; nb = du; }
            d = 0;
            bool big = false;
            for (uint32_t base = 0; base < nb; base += 32) {
                uint32_t j = base + lane;
                uint32_t x = j < nb ? B[j] : 0;
                bool hit = j < nb && find_sorted(A, 0, na, x) != NONE;
                unsigned bal = __ballot_sync(0xffffffffu, hit);
                uint32_t pos = d + __popc(bal & lanemask_lt());
                if (hit && pos < 32) ws.cand[pos] = x;
                d += __popc(bal);
                if (d > SMALL_D) { big = true; break; }
            }
            if (big) {
                if (lane == 0) P.defer_items[atomicAdd(P.defer_count, 1u)] = item;
                continue;
            }
            if (d + s0 < P.k || d == 0) continue;
        }
        __syncwarp();
        // rows: one per candidate, built cooperatively (lanes over N+(cand[i]))
        const uint32_t last = ws.cand[d - 1];
        for (uint32_t r = 0; r < d; ++r) {
            const uint32_t x = ws.cand[r];
            const uint32_t b = P.rp[x], e = P.rp[x + 1];
            uint32_t bits = 0;
            for (uint32_t j0 = b; j0 < e; j0 += 32) {
                uint32_t j = j0 + lane;
                uint32_t y = j < e ? P.col[j] : NONE;
                if (y != NONE && y <= last) {
                    uint32_t pos = find_sorted(ws.cand, r + 1, d, y);
                    if (pos != NONE) bits |= 1u << pos;
                }
                if (__shfl_sync(0xffffffffu, y, 31) >= last) break;
            }
            bits = __reduce_or_sync(0xffffffffu, bits);
            if (lane == 0) ws.row[r] = bits;
        }
        __syncwarp();
        // each lane walks the subtree below candidate `lane`
        if (lane < (int)d) {
            const uint32_t R = ws.row[lane];
            uint64_t c = 0;
            if (rem0 == 0) c = 1;
            else if (rem0 == 1) c = __popc(R);
            else if (rem0 == 2) c = edge_count1(R, ws.row);
            else if ((uint32_t)__popc(R) >= rem0) c = lane_walk(R, rem0, ws.row, ws.stk);
            acc_add(alo, ahi, c);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------

template <int G, bool EC, bool DO_BIG, bool DO_SMALL>
__global__ void __launch_bounds__(BLOCK) k_count_orient(const CountParams P) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ BlockShared sh;
    unsigned long long alo = 0, ahi = 0;
    if (DO_BIG) block_phase<G, EC>(P, smem, sh, alo, ahi);
    if (DO_SMALL) {
        WarpShared* ws = reinterpret_cast<WarpShared*>(smem) + (threadIdx.x >> 5);
        __syncthreads();
        warp_phase<EC>(P, *ws, alo, ahi);
    }
    // reduce: warp (exact 128-bit), then one atomic pair per warp
    unsigned long long hi_sum = ahi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, alo, o);
        unsigned long long yh = __shfl_xor_sync(0xffffffffu, hi_sum, o);
        unsigned long long s = alo + y;
        hi_sum += yh + (s < alo ? 1ull : 0ull);
        alo = s;
    }
    if ((threadIdx.x & 31) == 0) {
        add_u128(&P.ctl->total_lo, &P.ctl->total_hi, alo);
        if (hi_sum) atomicAdd(&P.ctl->total_hi, hi_sum);
    }
}

__global__ void k_finalize(const Ctl* ctl, kc_result* out) {
    kc_result r;
    r.total = ctl->total_lo;
    r.total_hi = ctl->total_hi;
    r.flags = ctl->flags | (ctl->total_hi ? KC_FLAG_TOTAL_OVERFLOW : 0u);
    r.status = (ctl->flags & KC_FLAG_TIMEOUT) ? KC_E_TIMEOUT : ((ctl->flags & KC_FLAG_INTERNAL) ? KC_E_INTERNAL : KC_OK);
    *out = r;
}

__global__ void k_write_result(kc_result* out, unsigned long long lo) {
    kc_result r;
    r.total = lo;
    r.total_hi = 0;
    r.flags = 0;
    r.status = KC_OK;
    *out = r;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef void (*CountKernel)(const CountParams);

template <int G, bool EC, bool B, bool S>
static CountKernel pick3() { return k_count_orient<G, EC, B, S>; }

template <bool EC, bool B, bool S>
static CountKernel pick2(uint32_t G) {
    switch (G) {
        case 1: return pick3<1, EC, B, S>();
        case 2: return pick3<2, EC, B, S>();
        case 4: return pick3<4, EC, B, S>();
        case 8: return pick3<8, EC, B, S>();
        case 16: return pick3<16, EC, B, S>();
        default: return pick3<32, EC, B, S>();
    }
}

static CountKernel pick_kernel(uint32_t G, bool ec, bool big, bool small) {
    if (!ec) {
        if (big && small) return pick2<false, true, true>(G);
        if (big) return pick2<false, true, false>(G);
        return pick2<false, false, true>(G);
    }
    if (big) return pick2<true, true, false>(G);
    return pick2<true, false, true>(G);
}

static constexpr size_t SMEM_LIMIT = 220 * 1024;

struct Geometry {
    uint32_t dcap, wcap, depth;
    int bitmap_in_smem, stack_in_smem;
    size_t smem_bytes;
    size_t gscratch_words;
};

static Geometry plan_geometry(uint32_t dcap, uint32_t k, uint32_t G, bool ec) {
    Geometry g;
    g.dcap = dcap < 1 ? 1 : dcap;
    g.wcap = (g.dcap + 31) / 32;
    const uint32_t s0 = ec ? 2 : 1;
    // stack levels: the DFS pushes while rem >= 3, i.e. rem0 - 2 levels
    uint32_t rem0 = k > s0 + 1 ? k - s0 - 1 : 0;
    g.depth = rem0 > 2 ? rem0 - 2 : 1;
    size_t cand_w = (g.dcap + 31) & ~31u;
    size_t bm_w = (size_t)g.dcap * g.wcap;
    size_t stk_w = (size_t)(BLOCK / G) * g.depth * g.wcap;
    size_t warp_bytes = sizeof(WarpShared) * NWARPS;
    size_t all = (cand_w + bm_w + stk_w) * 4;
    if (all <= SMEM_LIMIT) {
        g.bitmap_in_smem = 1;
        g.stack_in_smem = 1;
        g.smem_bytes = all;
        g.gscratch_words = 0;
    } else if ((cand_w + bm_w) * 4 <= SMEM_LIMIT) {
        g.bitmap_in_smem = 1;
        g.stack_in_smem = 0;
        g.smem_bytes = (cand_w + bm_w) * 4;
        g.gscratch_words = stk_w;
    } else {
        g.bitmap_in_smem = 0;
        g.stack_in_smem = 0;
        g.smem_bytes = cand_w * 4;
        g.gscratch_words = bm_w + stk_w;
    }
    if (g.smem_bytes < warp_bytes) g.smem_bytes = warp_bytes;
    g.gscratch_words = (g.gscratch_words + 63) & ~(size_t)63;
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

kc_status count_reserve(kc_graph* g, uint32_t k_max, int pivot, int per_vertex, cudaStream_t s) {
    (void)pivot;
    (void)per_vertex;
    (void)s;
    KC_CHECK(dev_alloc(g->ctl, sizeof(Ctl) + 256));
    Geometry geo = plan_geometry(g->d_max, k_max, 1, false);
    int blocks = g->sm_count * 8;
    KC_CHECK(dev_alloc(g->scratch, (geo.gscratch_words * blocks + 64) * 4));
    if (g->m) KC_CHECK(ensure_edge_src(g, s));
    return KC_OK;
}

kc_status count_launch(kc_graph* g, const CountArgs& a, kc_result* result_dev, cudaStream_t s) {
    const uint32_t k = a.k;
    KC_CHECK(dev_alloc(g->ctl, sizeof(Ctl) + 256));
    Ctl* ctl = (Ctl*)g->ctl.ptr;
    KC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    if (k <= 2 || (uint64_t)k > (uint64_t)g->d_max + 1) {
        unsigned long long v = k == 1 ? g->n : (k == 2 ? g->m : 0ull);
        k_write_result<<<1, 1, 0, s>>>(result_dev, v);
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    const bool ec = a.scheme == KC_SCHEME_EC;
    const uint32_t G = a.subwarp;
    if (k > MAX_DEPTH + 4)
        return set_error(KC_E_UNSUPPORTED, "orientation traversal supports k <= %d; use pivoting for larger k",
                         MAX_DEPTH + 4);
    CountParams P;
    memset(&P, 0, sizeof(P));
    P.rp = (const uint32_t*)g->row_ptr.ptr;
    P.col = (const uint32_t*)g->col.ptr;
    P.n = g->n;
    P.k = k;
    P.ctl = ctl;
    const int sms = g->sm_count;
    if (!ec) {
        // roots sorted by out-degree, descending; only those with d >= k-1 can hold a k-clique
        uint64_t n_work = roots_with_outdeg_at_least(g, k - 1);
        uint64_t n_big = roots_with_outdeg_at_least(g, (uint64_t)SMALL_D + 1 > k - 1 ? SMALL_D + 1 : k - 1);
        Geometry geo = plan_geometry(g->d_max, k, G, false);
        P.big_items = (const uint32_t*)g->roots.ptr;
        P.big_count = (uint32_t)n_big;
        P.small_items = (const uint32_t*)g->roots.ptr + n_big;
        P.small_count = (uint32_t)(n_work - n_big);
        P.dcap = geo.dcap;
        P.wcap = geo.wcap;
        P.depth = geo.depth;
        P.bitmap_in_smem = geo.bitmap_in_smem;
        P.stack_in_smem = geo.stack_in_smem;
        CountKernel kern = pick_kernel(G, false, n_big > 0, true);
        KC_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem_bytes));
        int bps = 0;
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BLOCK, geo.smem_bytes));
        if (bps < 1) return set_error(KC_E_UNSUPPORTED, "count kernel cannot be resident (smem %zu)", geo.smem_bytes);
        int blocks = bps * sms;
        KC_CHECK(dev_alloc(g->scratch, (geo.gscratch_words * blocks + 64) * 4));
        P.gscratch = (uint32_t*)g->scratch.ptr;
        P.gscratch_words = geo.gscratch_words;
        if (n_work > 0) {
            kern<<<blocks, BLOCK, geo.smem_bytes, s>>>(P);
            KC_CUDA(cudaGetLastError());
        }
    } else {
        KC_CHECK(ensure_edge_src(g, s));
        Geometry geo = plan_geometry(g->d_max, k, G, true);
        P.edge_src = (const uint32_t*)g->edge_src.ptr;
        P.dcap = geo.dcap;
        P.wcap = geo.wcap;
        P.depth = geo.depth;
        P.bitmap_in_smem = geo.bitmap_in_smem;
        P.stack_in_smem = geo.stack_in_smem;
        // phase 1: every edge in warp mode; bigger candidate sets are deferred
        KC_CHECK(dev_alloc(g->tmp, (size_t)g->m * 4 + 256));
        uint32_t* deferred = (uint32_t*)g->tmp.ptr;
        P.small_items = (const uint32_t*)g->edge_order.ptr;
        P.small_count = (uint32_t)g->m;
        P.defer_items = deferred;
        P.defer_count = &ctl->work_next_aux;
        CountKernel k1 = pick_kernel(G, true, false, true);
        KC_CUDA(cudaFuncSetAttribute((const void*)k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(WarpShared) * NWARPS)));
        int bps1 = 0;
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps1, k1, BLOCK, sizeof(WarpShared) * NWARPS));
        if (bps1 < 1) bps1 = 1;
        if (g->m > 0) {
            k1<<<bps1 * sms, BLOCK, sizeof(WarpShared) * NWARPS, s>>>(P);
            KC_CUDA(cudaGetLastError());
        }
        // phase 2: deferred edges in block mode (count read on the device)
        CountParams P2 = P;
        P2.small_items = nullptr;
        P2.small_count = 0;
        P2.big_items = deferred;
        P2.big_count_dev = &ctl->work_next_aux;
        CountKernel k2 = pick_kernel(G, true, true, false);
        KC_CUDA(cudaFuncSetAttribute((const void*)k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem_bytes));
        int bps = 0;
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k2, BLOCK, geo.smem_bytes));
        if (bps < 1) return set_error(KC_E_UNSUPPORTED, "count kernel cannot be resident (smem %zu)", geo.smem_bytes);
        int blocks = bps * sms;
        KC_CHECK(dev_alloc(g->scratch, (geo.gscratch_words * blocks + 64) * 4));
        P2.gscratch = (uint32_t*)g->scratch.ptr;
        P2.gscratch_words = geo.gscratch_words;
        if (g->m > 0) {
            k2<<<blocks, BLOCK, geo.smem_bytes, s>>>(P2);
            KC_CUDA(cudaGetLastError());
        }
    }
    k_finalize<<<1, 1, 0, s>>>(ctl, result_dev);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

}  // namespace kc
