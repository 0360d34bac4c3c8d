// Errors, device buffers and small host<->device helpers.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace csl {

thread_local std::string t_last_error;

void set_last_error(const std::string& m) { t_last_error = m; }
const char* last_error_cstr() { return t_last_error.c_str(); }

void fail(csl_status code, const std::string& msg) { throw Error(code, msg); }

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) throw Error(CSL_ERR_OOM, m);
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        throw Error(CSL_ERR_NOT_READY, m);
    throw Error(CSL_ERR_CUDA, m);
}

namespace {
std::atomic<int64_t> g_live{0}, g_peak{0};
thread_local int64_t t_launches = 0;
}

void launched(const char* what) {
    ++t_launches;
    check_cuda(cudaGetLastError(), what);
}

int64_t launches_and_reset() {
    int64_t n = t_launches;
    t_launches = 0;
    return n;
}

void note_device_bytes(int64_t delta) {
    int64_t v = g_live.fetch_add(delta) + delta;
    int64_t p = g_peak.load();
    while (v > p && !g_peak.compare_exchange_weak(p, v)) {
    }
}

int64_t device_bytes_peak_and_reset() {
    int64_t p = g_peak.exchange(g_live.load());
    return p;
}

[[noreturn]] static void alloc_error(cudaError_t e, size_t bytes) {
    cudaGetLastError();
    std::string m = "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                    cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) throw Error(CSL_ERR_OOM, m);
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        throw Error(CSL_ERR_NOT_READY, m);
    throw Error(CSL_ERR_CUDA, m);
}

// Keep freed workspace in the stream-ordered pool instead of returning it to
// the driver at every synchronisation (per process, per device).
static void keep_pool_memory() {
    static thread_local int done_for = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev == done_for) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done_for = dev;
}

void DevBuf::alloc(size_t bytes, cudaStream_t s) {
    release();
    keep_pool_memory();
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) alloc_error(e, bytes);
    p_ = p;
    n_ = bytes;
    s_ = s;
    persistent_ = false;
    note_device_bytes((int64_t)bytes);
}

void DevBuf::alloc_persistent(size_t bytes) {
    release();
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) alloc_error(e, bytes);
    p_ = p;
    n_ = bytes;
    s_ = nullptr;
    persistent_ = true;
    note_device_bytes((int64_t)bytes);
}

void DevBuf::release() {
    if (!p_) return;
    if (persistent_) cudaFree(p_);
    else cudaFreeAsync(p_, s_);
    note_device_bytes(-(int64_t)n_);
    p_ = nullptr;
    n_ = 0;
}

void read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    CSL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    CSL_CUDA(cudaStreamSynchronize(s));
}

int64_t read_i64(const int64_t* dev, cudaStream_t s) {
    int64_t v = 0;
    read_to_host(&v, dev, sizeof(v), s);
    return v;
}

}  // namespace csl
