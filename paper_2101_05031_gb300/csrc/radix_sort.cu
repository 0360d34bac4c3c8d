// Stable least-significant-digit radix sort of (uint32 key, uint32 value)
// pairs, 8 bits per pass. Each pass: a per-tile digit histogram, a
// device-wide scan of the digit-major histogram table, then a scatter in
// which every element's rank inside its tile is computed in input order, so
// equal keys keep their input order (the sort is deterministic).
#include "common.cuh"

namespace csl {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kThreads) k_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                   int shift, uint32_t* __restrict__ hist,
                                                   int64_t n_tiles) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + (int64_t)i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    // digit-major: all tiles of digit 0, then digit 1, ...
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint32_t* __restrict__ keys_in,
                                                      const uint32_t* __restrict__ vals_in,
                                                      uint32_t* __restrict__ keys_out,
                                                      uint32_t* __restrict__ vals_out, int64_t n,
                                                      int shift,
                                                      const uint32_t* __restrict__ hist_scan,
                                                      int64_t n_tiles) {
    __shared__ uint32_t run[kRadix];            // elements of each digit placed so far
    __shared__ uint32_t wcnt[kWarps][kRadix];   // this round: per-warp counts -> offsets
    __shared__ uint32_t gbase[kRadix];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    gbase[threadIdx.x] = hist_scan[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int i = 0; i < kItems; ++i) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t idx = base + (int64_t)i * kThreads + threadIdx.x;
        bool valid = idx < n;
        uint32_t key = valid ? keys_in[idx] : 0u;
        uint32_t val = valid ? vals_in[idx] : 0u;
        // invalid lanes get a digit of their own (256) that matches no real one
        uint32_t digit = valid ? ((key >> shift) & 0xffu) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        unsigned rank_in_warp = __popc(peers & lt_mask);
        bool leader = (peers & lt_mask) == 0;
        if (valid && leader) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive offsets over the warps of this round
            int d = threadIdx.x;
            uint32_t acc = run[d];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                uint32_t c = wcnt[w][d];
                wcnt[w][d] = acc;
                acc += c;
            }
            run[d] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = gbase[digit] + wcnt[warp][digit] + rank_in_warp;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

}  // namespace

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tmp_keys, uint32_t* tmp_vals,
                      int64_t n, int key_bits, cudaStream_t s) {
    if (n <= 1 || key_bits <= 0) return;
    if (n > (int64_t)0xffffffffLL) fail(CSL_ERR_CAPACITY, "radix sort: more than 2^32 elements");
    int64_t n_tiles = ceil_div(n, kTile);
    DevBuf hist((size_t)kRadix * n_tiles * sizeof(uint32_t), s);
    int passes = (key_bits + 7) / 8;
    uint32_t *ki = keys, *vi = vals, *ko = tmp_keys, *vo = tmp_vals;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_hist<<<(unsigned)n_tiles, kThreads, 0, s>>>(ki, n, shift, hist.as<uint32_t>(), n_tiles);
        CSL_LAUNCH_CHECK("radix hist");
        exclusive_scan_u32(hist.as<uint32_t>(), hist.as<uint32_t>(), kRadix * n_tiles, nullptr, s);
        k_scatter<<<(unsigned)n_tiles, kThreads, 0, s>>>(ki, vi, ko, vo, n, shift,
                                                         hist.as<uint32_t>(), n_tiles);
        CSL_LAUNCH_CHECK("radix scatter");
        uint32_t* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (ki != keys) {   // odd number of passes: copy back
        CSL_CUDA(cudaMemcpyAsync(keys, ki, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        CSL_CUDA(cudaMemcpyAsync(vals, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace csl
