// Device-wide exclusive prefix sums (reduce, scan the block sums, scan again
// with the block's offset). A block of 256 threads takes a tile of 2048
// elements, 8 consecutive ones per thread, moved as 16-byte vectors.
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

// Thread t of a block owns the kItems consecutive elements base + t * kItems ...
// of the block's tile: loaded as 16-byte vectors when the tile is whole and
// aligned (a warp then reads 32 consecutive 16-byte pieces per vector load).
template <class T>
__device__ __forceinline__ void load_items(const T* __restrict__ in, int64_t n, int64_t first,
                                           T (&v)[kItems]) {
    static_assert((kItems * sizeof(T)) % 16 == 0, "whole vectors per thread");
    if (first + kItems <= n && (reinterpret_cast<uintptr_t>(in + first) & 15) == 0) {
        const uint4* p = reinterpret_cast<const uint4*>(in + first);
#pragma unroll
        for (int q = 0; q < (int)(kItems * sizeof(T) / 16); ++q)
            reinterpret_cast<uint4*>(v)[q] = __ldg(p + q);
    } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i) v[i] = first + i < n ? in[first + i] : (T)0;
    }
}

template <class U>
__device__ __forceinline__ void store_items(U* __restrict__ out, int64_t n, int64_t first,
                                            const U (&v)[kItems]) {
    if (first + kItems <= n && (reinterpret_cast<uintptr_t>(out + first) & 15) == 0 &&
        (kItems * sizeof(U)) % 16 == 0) {
        uint4* p = reinterpret_cast<uint4*>(out + first);
#pragma unroll
        for (int q = 0; q < (int)(kItems * sizeof(U) / 16); ++q)
            p[q] = reinterpret_cast<const uint4*>(v)[q];
    } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (first + i < n) out[first + i] = v[i];
    }
}

// Exclusive block-wide scan of one value per thread; the block total goes to
// *total_s (shared), visible to every thread on return.
template <class U>
__device__ __forceinline__ U block_exclusive(U x, U* total_s) {
    __shared__ U warp_tot[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const U inc = warp_inclusive(x, lane);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const U t = lane < kThreads / 32 ? warp_tot[lane] : (U)0;
        const U ti = warp_inclusive(t, lane);
        if (lane < kThreads / 32) warp_tot[lane] = ti - t;   // exclusive warp offsets
        if (lane == kThreads / 32 - 1) *total_s = ti;
    }
    __syncthreads();
    return warp_tot[warp] + inc - x;
}

template <class T, class U>
__global__ void __launch_bounds__(kThreads) k_block_sums(const T* __restrict__ in, int64_t n,
                                                         U* __restrict__ sums) {
    __shared__ U warp_tot[kThreads / 32];
    T v[kItems];
    load_items(in, n, (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems, v);
    U acc = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) acc += (U)v[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    __shared__ U block_total;
    const int64_t first = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    T v[kItems];
    load_items(in, n, first, v);
    U mine = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) mine += (U)v[i];
    const U off = block_exclusive<U>(mine, &block_total);
    const U carry = offsets ? offsets[blockIdx.x] : (U)0;
    U r[kItems];
    U run = carry + off;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        r[i] = run;
        run += (U)v[i];
    }
    store_items(out, n, first, r);
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = carry + block_total;
}

// Flag counts per tile, the flag being the top bit of each word.
__global__ void __launch_bounds__(kThreads) k_flag_sums(const uint32_t* __restrict__ in, int64_t n,
                                                        uint32_t* __restrict__ sums) {
    __shared__ uint32_t warp_tot[kThreads / 32];
    uint32_t v[kItems];
    load_items(in, n, (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems, v);
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) acc += v[i] >> 31;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) warp_tot[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += warp_tot[w];
        sums[blockIdx.x] = t;
    }
}

// pos: exclusive scan of the flags of one tile per block (plus the tile's
// offset); list[pos[i]] = i for every flagged i.
__global__ void __launch_bounds__(kThreads) k_flag_scan_list(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ pos, int64_t n,
                                                             const uint32_t* __restrict__ offsets,
                                                             uint32_t* __restrict__ list,
                                                             int64_t list_cap, uint32_t* total,
                                                             uint32_t* status) {
    __shared__ uint32_t block_total;
    const int64_t first = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    uint32_t v[kItems];
    load_items(in, n, first, v);
    uint32_t mine = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) mine += v[i] >> 31;
    const uint32_t off = block_exclusive<uint32_t>(mine, &block_total);
    const uint32_t carry = offsets ? offsets[blockIdx.x] : 0u;
    uint32_t r[kItems];
    uint32_t run = carry + off;
    bool over = false;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        r[i] = run;
        if ((v[i] >> 31) && first + i < n) {
            if ((int64_t)run < list_cap) list[run] = (uint32_t)(first + i);
            else over = true;
        }
        run += v[i] >> 31;
    }
    store_items(pos, n, first, r);
    if (over) atomicOr(status, ST_CAPACITY);
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = carry + block_total;
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

void scan_flags_list(const uint32_t* word, int64_t n, uint32_t* pos, uint32_t* list,
                     int64_t list_cap, uint32_t* total_dev, uint32_t* status, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) CSL_CUDA(cudaMemsetAsync(total_dev, 0, 4, s));
        return;
    }
    const int64_t nb = ceil_div(n, kTile);
    DevBuf sums((size_t)nb * 4, s);
    if (nb > 1) {
        k_flag_sums<<<(unsigned)nb, kThreads, 0, s>>>(word, n, sums.as<uint32_t>());
        CSL_LAUNCH_CHECK("flag sums");
        scan_impl<uint32_t, uint32_t>(sums.as<uint32_t>(), sums.as<uint32_t>(), nb, nullptr, s);
    }
    k_flag_scan_list<<<(unsigned)nb, kThreads, 0, s>>>(word, pos, n,
                                                       nb > 1 ? sums.as<uint32_t>() : nullptr,
                                                       list, list_cap, total_dev, status);
    CSL_LAUNCH_CHECK("flag scan");
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
