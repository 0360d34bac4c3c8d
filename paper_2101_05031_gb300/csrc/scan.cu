// Device-wide exclusive prefix sums (reduce, scan the block sums, scan again
// with the block's offset). Blocks of 256 threads take 8 consecutive segments
// of 256 elements each; every global load and store is coalesced.
#include "common.cuh"

namespace csl {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <class U>
__device__ __forceinline__ U warp_inclusive(U v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        U t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

template <class T, class U>
__global__ void __launch_bounds__(kThreads) k_block_sums(const T* __restrict__ in, int64_t n,
                                                         U* __restrict__ sums) {
    __shared__ U warp_tot[kThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kTile;
    U acc = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + (int64_t)i * kThreads + threadIdx.x;
        if (idx < n) acc += (U)in[idx];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) warp_tot[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        U t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += warp_tot[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive scan of one tile per block, plus the block's offset (if any).
template <class T, class U>
__global__ void __launch_bounds__(kThreads) k_block_scan(const T* in, U* out, int64_t n,
                                                         const U* __restrict__ offsets,
                                                         U* total) {
    __shared__ U warp_tot[kThreads / 32];
    __shared__ U carry_s;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t base = (int64_t)blockIdx.x * kTile;
    U carry = offsets ? offsets[blockIdx.x] : (U)0;
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = base + (int64_t)i * kThreads + threadIdx.x;
        U v = idx < n ? (U)in[idx] : (U)0;
        U inc = warp_inclusive(v, lane);
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            U t = lane < kThreads / 32 ? warp_tot[lane] : (U)0;
            U ti = warp_inclusive(t, lane);
            if (lane < kThreads / 32) warp_tot[lane] = ti - t;      // exclusive warp offsets
            if (lane == kThreads / 32 - 1) carry_s = ti;             // tile segment total
        }
        __syncthreads();
        U res = carry + warp_tot[warp] + inc - v;
        U seg = carry_s;
        __syncthreads();   // warp_tot / carry_s are rewritten next iteration
        if (idx < n) out[idx] = res;
        carry += seg;
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = carry;
}

template <class T, class U>
void scan_impl(const T* in, U* out, int64_t n, U* total_dev, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) CSL_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(U), s));
        return;
    }
    int64_t nb = ceil_div(n, kTile);
    if (nb == 1) {
        k_block_scan<T, U><<<1, kThreads, 0, s>>>(in, out, n, nullptr, total_dev);
        CSL_LAUNCH_CHECK("scan");
        return;
    }
    DevBuf sums((size_t)nb * sizeof(U), s);
    k_block_sums<T, U><<<(unsigned)nb, kThreads, 0, s>>>(in, n, sums.as<U>());
    CSL_LAUNCH_CHECK("scan sums");
    scan_impl<U, U>(sums.as<U>(), sums.as<U>(), nb, total_dev, s);
    k_block_scan<T, U><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, sums.as<U>(), nullptr);
    CSL_LAUNCH_CHECK("scan tiles");
}

}  // namespace

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                        cudaStream_t s) {
    scan_impl<uint32_t, uint32_t>(in, out, n, total_dev, s);
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                        cudaStream_t s) {
    scan_impl<int64_t, int64_t>(in, out, n, total_dev, s);
}

void exclusive_scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                               cudaStream_t s) {
    scan_impl<uint32_t, int64_t>(in, out, n, total_dev, s);
}

}  // namespace csl
