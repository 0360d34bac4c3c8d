// Errors, device buffers and small host<->device helpers.
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>
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

int64_t device_bytes_live() { return g_live.load(); }
int64_t device_bytes_peak() { return g_peak.load(); }

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
// the CUDA driver at every synchronisation (per process, per device).
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
    keep_pool_memory();
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    // From the stream-ordered pool too (what a freed lattice or batch left
    // there is reused without a round trip to the driver, which maps every
    // page again): ordered on the legacy default stream and complete before
    // this returns, so that any stream may use it.
    cudaError_t e = cudaMallocAsync(&p, bytes, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) alloc_error(e, bytes);
    p_ = p;
    n_ = bytes;
    s_ = nullptr;
    persistent_ = true;
    note_device_bytes((int64_t)bytes);
}

void DevBuf::release() {
    if (!p_) return;
    if (!owned_) {   // a view of memory owned elsewhere
        p_ = nullptr;
        n_ = 0;
        owned_ = true;
        return;
    }
    if (persistent_) {   // any stream may still use it: wait for the device, as cudaFree does
        cudaDeviceSynchronize();
        cudaFreeAsync(p_, 0);
    } else {
        cudaFreeAsync(p_, s_);
    }
    note_device_bytes(-(int64_t)n_);
    p_ = nullptr;
    n_ = 0;
}

void DevBuf::view(void* p, size_t bytes) {
    release();
    p_ = p;
    n_ = bytes;
    owned_ = false;
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

void* host_block_take_largest(size_t* bytes) {
    std::lock_guard<std::mutex> lk(g_host_mu);
    if (g_host_free.empty()) {
        *bytes = 0;
        return nullptr;
    }
    auto it = std::prev(g_host_free.end());
    void* p = it->second;
    *bytes = it->first;
    g_host_free_bytes -= it->first;
    g_host_free.erase(it);
    return p;
}

size_t vertex_block_eid_offset(size_t block_bytes, bool want_eid) {
    // 8 bytes of xy and 4 of edge id per vertex: the edge ids start at 2/3
    return want_eid ? ((block_bytes / 12) * 8 + 15) & ~(size_t)15 : block_bytes;
}

csl_contours* new_host_contours(int32_t n_layers, int64_t n_loops, int64_t n_verts, bool want_eid,
                                void* vertex_block) {
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t b0 = up16((size_t)(n_layers + 1) * 8), b1 = up16((size_t)(n_loops + 1) * 8);
    char* offs = static_cast<char*>(host_block_alloc(b0 + b1));
    char* verts = static_cast<char*>(vertex_block);
    if (!verts) {
        try {
            const size_t vb = (size_t)n_verts * (want_eid ? 12 : 8) + 32;
            verts = static_cast<char*>(host_block_alloc(vb));
        } catch (...) {
            host_block_free(offs);
            throw;
        }
    }
    csl_contours* c = new (std::nothrow) csl_contours();
    if (!c) {
        host_block_free(offs);
        if (!vertex_block) host_block_free(verts);
        fail(CSL_ERR_OOM, "host allocation failed");
    }
    memset(c, 0, sizeof(*c));
    c->n_layers = n_layers;
    c->on_device = 0;
    c->n_loops = n_loops;
    c->n_verts = n_verts;
    c->layer_loop_off = reinterpret_cast<int64_t*>(offs);
    c->loop_vert_off = reinterpret_cast<int64_t*>(offs + b0);
    c->xy = reinterpret_cast<float*>(verts);
    if (want_eid) {
        // the edge ids follow the vertices in the same block
        size_t bytes = 0;
        {
            std::lock_guard<std::mutex> lk(g_host_mu);
            auto it = g_host_pinned.find(verts);
            bytes = it != g_host_pinned.end() ? it->second : (size_t)n_verts * 12 + 32;
        }
        c->edge_id = reinterpret_cast<int32_t*>(verts + vertex_block_eid_offset(bytes, true));
    }
    return c;
}

// Small read-backs go through a kernel that stores into page-locked host
// memory, not through a copy engine: a copy engine may be busy with a large
// device-to-host transfer of results on another stream, and a small copy
// queued behind it would stall the host for the duration of that transfer.
__global__ void k_read_back(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                            int n_words) {
    for (int i = threadIdx.x; i < n_words; i += blockDim.x) dst[i] = src[i];
}

namespace {
constexpr size_t kReadBackBytes = 64 << 10;
// (host pointer, device pointer) of this host thread's buffer, kept for the
// thread's lifetime; {nullptr, nullptr} when page-locked memory is unavailable.
std::pair<uint32_t*, uint32_t*> read_back_buffer() {
    static thread_local uint32_t* host = nullptr;
    static thread_local uint32_t* dev = nullptr;
    if (!host) {
        void* p = nullptr;
        void* d = nullptr;
        if (cudaHostAlloc(&p, kReadBackBytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess) {
            cudaGetLastError();
            return {nullptr, nullptr};
        }
        if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(p);
            return {nullptr, nullptr};
        }
        host = static_cast<uint32_t*>(p);
        dev = static_cast<uint32_t*>(d);
    }
    return {host, dev};
}
}  // namespace

void read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    std::pair<uint32_t*, uint32_t*> buf{nullptr, nullptr};
    if (bytes <= kReadBackBytes && bytes % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 4 == 0)
        buf = read_back_buffer();
    if (buf.first) {
        k_read_back<<<1, 256, 0, s>>>(static_cast<const uint32_t*>(src), buf.second,
                                      (int)(bytes / 4));
        CSL_LAUNCH_CHECK("read back");
        CSL_CUDA(cudaStreamSynchronize(s));
        memcpy(dst, buf.first, bytes);
        return;
    }
    CSL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    CSL_CUDA(cudaStreamSynchronize(s));
}

int64_t read_i64(const int64_t* dev, cudaStream_t s) {
    int64_t v = 0;
    read_to_host(&v, dev, sizeof(v), s);
    return v;
}

}  // namespace csl
