// Errors, device buffers and small host<->device helpers.
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

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

namespace {
std::mutex g_host_mu;
std::multimap<size_t, void*> g_host_free;           // cached page-locked blocks by size
std::unordered_map<void*, size_t> g_host_pinned;    // every page-locked block we own
size_t g_host_free_bytes = 0;
constexpr size_t kHostCacheCap = (size_t)64 << 30;   // free bytes kept for reuse
}  // namespace

void* host_block_alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_free.lower_bound(bytes);
        // reuse a cached block unless it is much larger than the request
        if (it != g_host_free.end() && it->first <= std::max(2 * bytes, bytes + ((size_t)64 << 20))) {
            void* p = it->second;
            g_host_free_bytes -= it->first;
            g_host_free.erase(it);
            return p;
        }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_host_mu);
        g_host_pinned[p] = bytes;
        return p;
    }
    cudaGetLastError();
    p = malloc(bytes);
    if (!p) fail(CSL_ERR_OOM, "host allocation of " + std::to_string(bytes) + " bytes failed");
    return p;
}

void host_block_free(void* p) {
    if (!p) return;
    std::vector<void*> drop;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_pinned.find(p);
        if (it == g_host_pinned.end()) {
            free(p);
            return;
        }
        g_host_free.emplace(it->second, p);
        g_host_free_bytes += it->second;
        while (g_host_free_bytes > kHostCacheCap && !g_host_free.empty()) {
            auto big = std::prev(g_host_free.end());
            g_host_free_bytes -= big->first;
            g_host_pinned.erase(big->second);
            drop.push_back(big->second);
            g_host_free.erase(big);
        }
    }
    for (void* q : drop) cudaFreeHost(q);
}

csl_contours* new_host_contours(int32_t n_layers, int64_t n_loops, int64_t n_verts, bool want_eid) {
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t b0 = up16((size_t)(n_layers + 1) * 8), b1 = up16((size_t)(n_loops + 1) * 8);
    const size_t b2 = up16((size_t)n_verts * 8), b3 = want_eid ? up16((size_t)n_verts * 4) : 0;
    char* base = static_cast<char*>(host_block_alloc(b0 + b1 + b2 + b3));
    csl_contours* c = new (std::nothrow) csl_contours();
    if (!c) {
        host_block_free(base);
        fail(CSL_ERR_OOM, "host allocation failed");
    }
    memset(c, 0, sizeof(*c));
    c->n_layers = n_layers;
    c->on_device = 0;
    c->n_loops = n_loops;
    c->n_verts = n_verts;
    c->layer_loop_off = reinterpret_cast<int64_t*>(base);
    c->loop_vert_off = reinterpret_cast<int64_t*>(base + b0);
    c->xy = reinterpret_cast<float*>(base + b0 + b1);
    c->edge_id = want_eid ? reinterpret_cast<int32_t*>(base + b0 + b1 + b2) : nullptr;
    return c;
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
