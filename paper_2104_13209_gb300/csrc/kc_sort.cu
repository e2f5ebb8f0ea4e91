// Stable LSD radix sort of vertex ids by a u32 key (8-bit digits).  It turns
// an orientation key (degree, or the peel round of the k-core decomposition,
// Section 3.1) into the vertex order; ties keep ascending id, so the order is
// (key, id).  Each 512-element tile is ranked by one warp with match/ballot
// primitives, which keeps the scatter stable.
#include "kc_common.cuh"

namespace kc {

static constexpr int SORT_WARPS = 8;
static constexpr int SORT_ITEMS = 16;
static constexpr int SORT_TILE = 32 * SORT_ITEMS;  // elements per warp tile

// Pass input: key of element i is keys[i], or key_of_id of its id on the
// first pass (the id is vals[i], or i when vals is null).
__device__ __forceinline__ uint32_t load_key(const uint32_t* keys, const uint32_t* key_of_id, const uint32_t* vals,
                                             uint32_t i) {
    return keys ? keys[i] : key_of_id[vals ? vals[i] : i];
}

__global__ void __launch_bounds__(SORT_WARPS * 32) k_radix_hist(const uint32_t* __restrict__ keys,
                                                                const uint32_t* __restrict__ key_of_id,
                                                                const uint32_t* __restrict__ vals, uint32_t n,
                                                                int shift, uint32_t ntiles,
                                                                uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[SORT_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x * SORT_WARPS + w;
    for (int b = lane; b < 256; b += 32) h[w][b] = 0;
    __syncwarp();
    if (tile < ntiles) {
        for (int it = 0; it < SORT_ITEMS; ++it) {
            uint32_t i = tile * SORT_TILE + it * 32 + lane;
            if (i < n) atomicAdd(&h[w][(load_key(keys, key_of_id, vals, i) >> shift) & 255u], 1u);
        }
    }
    __syncwarp();
    if (tile < ntiles)
        for (int b = lane; b < 256; b += 32) hist[(size_t)b * ntiles + tile] = h[w][b];
}

__global__ void __launch_bounds__(SORT_WARPS * 32) k_radix_scatter(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ key_of_id, const uint32_t* __restrict__ vals,
    uint32_t n, int shift, uint32_t ntiles, const uint32_t* __restrict__ offs, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t run[SORT_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x * SORT_WARPS + w;
    if (tile >= ntiles) return;
    for (int b = lane; b < 256; b += 32) run[w][b] = offs[(size_t)b * ntiles + tile];
    __syncwarp();
    const unsigned lt = lanemask_lt();
    for (int it = 0; it < SORT_ITEMS; ++it) {
        uint32_t i = tile * SORT_TILE + it * 32 + lane;
        bool valid = i < n;
        uint32_t key = valid ? load_key(keys, key_of_id, vals, i) : 0u;
        uint32_t val = valid ? (vals ? vals[i] : i) : 0u;
        uint32_t d = valid ? ((key >> shift) & 255u) : (256u + lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t base = valid ? run[w][d] : 0u;
        __syncwarp();
        if (valid) {
            uint32_t pos = base + __popc(peers & lt);
            keys_out[pos] = key;
            vals_out[pos] = val;
            if ((peers & lt) == 0) run[w][d] = base + __popc(peers);
        }
        __syncwarp();
    }
}

kc_status sort_ids_by_key(const uint32_t* key, uint32_t n, uint32_t max_key, uint32_t* out_ids, DevBuf& tmp,
                          cudaStream_t s, const uint32_t* in_ids) {
    if (n == 0) return KC_OK;
    int passes = 1;
    while (passes < 4 && (max_key >> (8 * passes)) != 0) ++passes;
    const uint32_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    const size_t hist_n = (size_t)256 * ntiles;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t need = 4 * al((size_t)n * 4) + 2 * al((hist_n + 1) * 4) + al(scan_tmp_bytes(hist_n));
    KC_CHECK(dev_alloc(tmp, need));
    char* p = (char*)tmp.ptr;
    uint32_t* ka = (uint32_t*)p; p += al((size_t)n * 4);
    uint32_t* kb = (uint32_t*)p; p += al((size_t)n * 4);
    uint32_t* va = (uint32_t*)p; p += al((size_t)n * 4);
    uint32_t* vb = (uint32_t*)p; p += al((size_t)n * 4);
    uint32_t* hist = (uint32_t*)p; p += al((hist_n + 1) * 4);
    uint32_t* offs = (uint32_t*)p; p += al((hist_n + 1) * 4);
    void* stmp = p;
    const unsigned blocks = (ntiles + SORT_WARPS - 1) / SORT_WARPS;
    const uint32_t* kin = nullptr;  // first pass reads key[id]
    const uint32_t* vin = in_ids;   // first pass: the given ids, or 0..n-1
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        uint32_t* kout = (ps & 1) ? kb : ka;
        uint32_t* vout = (ps == passes - 1) ? out_ids : ((ps & 1) ? vb : va);
        k_radix_hist<<<blocks, SORT_WARPS * 32, 0, s>>>(kin, key, vin, n, shift, ntiles, hist);
        note_launch();
        KC_CUDA(cudaGetLastError());
        KC_CHECK(scan_u32_raw(hist, offs, hist_n, stmp, s));
        k_radix_scatter<<<blocks, SORT_WARPS * 32, 0, s>>>(kin, key, vin, n, shift, ntiles, offs, kout, vout);
        note_launch();
        KC_CUDA(cudaGetLastError());
        kin = kout;
        vin = vout;
    }
    return KC_OK;
}

}  // namespace kc
