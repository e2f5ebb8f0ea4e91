// Exclusive prefix sum of u32 arrays (reduce-then-scan over 2048-element
// tiles, recursive over tile sums).  Used to rebuild CSR row pointers after
// the orientation filter (Section 3.1: "histogram and exclusive scan") and to
// place keys in the radix sort.
#include "kc_common.cuh"

namespace kc {

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_sums, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const uint32_t* __restrict__ in, size_t n,
                                                              uint32_t* __restrict__ sums) {
    __shared__ uint32_t ws[SCAN_THREADS / 32];
    size_t base = (size_t)blockIdx.x * SCAN_TILE;
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        size_t i = base + (size_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// out[i] = offsets[tile] + exclusive prefix within the tile; the block that
// holds the last element also writes out[n].
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const uint32_t* __restrict__ in, size_t n,
                                                            const uint32_t* __restrict__ offsets,
                                                            uint32_t* __restrict__ out) {
    __shared__ uint32_t ws[SCAN_THREADS / 32];
    __shared__ uint32_t chunk_total;
    size_t base = (size_t)blockIdx.x * SCAN_TILE;
    uint32_t carry = offsets ? offsets[blockIdx.x] : 0u;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        size_t i = base + (size_t)j * SCAN_THREADS + threadIdx.x;
        uint32_t x = i < n ? in[i] : 0u;
        uint32_t ex = block_exclusive_scan(x, ws, &chunk_total);
        if (i < n) out[i] = carry + ex;
        if (i == n - 1) out[n] = carry + ex + x;
        __syncthreads();
        carry += chunk_total;
        __syncthreads();
    }
}

__global__ void k_write_zero_total(uint32_t* out) { out[0] = 0; }

size_t scan_tmp_bytes(size_t n) {
    size_t total = 0;
    while (n > (size_t)SCAN_TILE) {
        size_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
        total += (2 * nt + 1 + 64) * sizeof(uint32_t);
        n = nt;
    }
    return total + 256;
}

static kc_status scan_rec(const uint32_t* in, uint32_t* out, size_t n, char* tmp, cudaStream_t s) {
    if (n == 0) {
        k_write_zero_total<<<1, 1, 0, s>>>(out);
        note_launch();
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    size_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt == 1) {
        k_tile_scan<<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
        note_launch();
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    uint32_t* sums = (uint32_t*)tmp;
    uint32_t* offs = sums + nt;
    char* next = (char*)(offs + nt + 1 + 64);
    k_tile_reduce<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, sums);
    note_launch();
    KC_CUDA(cudaGetLastError());
    KC_CHECK(scan_rec(sums, offs, nt, next, s));
    k_tile_scan<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, offs, out);
    note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status scan_u32(const uint32_t* in, uint32_t* out, size_t n, DevBuf& tmp, cudaStream_t s) {
    KC_CHECK(dev_alloc(tmp, scan_tmp_bytes(n)));
    return scan_rec(in, out, n, (char*)tmp.ptr, s);
}

kc_status scan_u32_raw(const uint32_t* in, uint32_t* out, size_t n, void* tmp, cudaStream_t s) {
    return scan_rec(in, out, n, (char*)tmp, s);
}

}  // namespace kc
