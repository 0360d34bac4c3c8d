// Internal helpers shared by the translation units of libcslice.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/cslice.h"

namespace csl {

// A failure inside the library; converted to a csl_status at the ABI.
struct Error : std::runtime_error {
    csl_status code;
    Error(csl_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void fail(csl_status code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);

#define CSL_CUDA(call) ::csl::check_cuda((call), #call)
// Placed after every kernel launch: checks it and counts it.
#define CSL_LAUNCH_CHECK(what) ::csl::launched(what)
void launched(const char* what);
int64_t launches_and_reset();

// Stream-ordered device allocation that frees itself (cudaFreeAsync).
class DevBuf {
  public:
    DevBuf() = default;
    DevBuf(size_t bytes, cudaStream_t s) { alloc(bytes, s); }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept
        : p_(o.p_), n_(o.n_), s_(o.s_), persistent_(o.persistent_), owned_(o.owned_) {
        o.p_ = nullptr; o.n_ = 0; o.owned_ = true;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p_ = o.p_; n_ = o.n_; s_ = o.s_; persistent_ = o.persistent_; owned_ = o.owned_;
            o.p_ = nullptr; o.n_ = 0; o.owned_ = true;
        }
        return *this;
    }
    // stream-ordered (cudaMallocAsync / cudaFreeAsync on the same stream)
    void alloc(size_t bytes, cudaStream_t s);
    void ensure(size_t bytes, cudaStream_t s) { if (bytes > n_) alloc(bytes, s); }
    // outlives any stream (from the same pool, allocated on the legacy stream and
    // synchronised; freed after a device synchronisation): for objects handed
    // to the caller
    void alloc_persistent(size_t bytes);
    void ensure_persistent(size_t bytes) { if (bytes > n_) alloc_persistent(bytes); }
    void release();
    // a view of `bytes` of device memory owned elsewhere (never freed here)
    void view(void* p, size_t bytes);
    template <class T> T* as() const { return reinterpret_cast<T*>(p_); }
    size_t size() const { return n_; }
    void* get() const { return p_; }

  private:
    void* p_ = nullptr;
    size_t n_ = 0;
    cudaStream_t s_ = nullptr;
    bool persistent_ = false;
    bool owned_ = true;
};

// A device array that grows in place (growmap.cu): reserve() takes a range of
// virtual addresses, ensure(n) maps physical memory behind its first n bytes
// (the base address never moves). hand_over() passes the memory to a registry
// from which growmap_free(base) releases it (csl_contours_free); otherwise the
// destructor releases it. Both wait for the device first.
class GrowMap {
  public:
    GrowMap() = default;
    ~GrowMap();
    GrowMap(const GrowMap&) = delete;
    GrowMap& operator=(const GrowMap&) = delete;
    void reserve(size_t bytes);
    void ensure(size_t bytes);
    void* base() const { return reinterpret_cast<void*>(va_); }
    void* hand_over();

  private:
    void free_all();
    unsigned long long va_ = 0;
    size_t reserved_ = 0, mapped_ = 0, gran_ = 0;
    int dev_ = 0;
    std::vector<std::pair<unsigned long long, size_t>> handles_;   // (handle, bytes)
};
bool growmap_available();
bool growmap_free(void* base);   // true when base came from hand_over()

// Workspace accounting for csl_last_stats.
void note_device_bytes(int64_t delta);
int64_t device_bytes_peak_and_reset();
int64_t device_bytes_live();   // bytes held now
int64_t device_bytes_peak();   // the peak since the last reset

void set_last_error(const std::string& m);
const char* last_error_cstr();

// Host memory for results handed to the caller: page-locked blocks (so that
// device-to-host copies run at the link's speed) kept in a per-process cache
// and reused by later results once the caller frees them. Falls back to
// malloc when page-locked memory cannot be had. Thread-safe.
void* host_block_alloc(size_t bytes);
void host_block_free(void* p);

// Takes the largest cached free block out of the cache (nullptr if none).
void* host_block_take_largest(size_t* bytes);

// Host contours in two host blocks: [layer_loop_off | loop_vert_off] and the
// vertex block [xy ... | edge_id ...] (edge ids from vertex_block_eid_offset);
// csl_contours_free releases both (their bases are layer_loop_off and xy).
// vertex_block: a block the vertices were already copied into (taken from the
// cache, large enough), or nullptr to allocate one.
size_t vertex_block_eid_offset(size_t block_bytes, bool want_eid);
csl_contours* new_host_contours(int32_t n_layers, int64_t n_loops, int64_t n_verts, bool want_eid,
                                void* vertex_block = nullptr);

int64_t read_i64(const int64_t* dev, cudaStream_t s);   // synchronising
void read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t s);  // synchronising

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline unsigned grid_for(int64_t n, int block, int64_t cap = 152 * 64) {
    int64_t g = ceil_div(n, block);
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ---- scan (scan.cu) ----
// Exclusive prefix sums; `out` may alias `in`. The total is written to
// *total_dev when it is non-null.
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                        cudaStream_t s);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                        cudaStream_t s);
// Numbering of flagged items, the flag being the top bit of word[i]:
// pos[i] = flagged items before i (every i), list[pos[i]] = i for flagged i
// (while pos[i] < list_cap; beyond it *status |= ST_CAPACITY), *total_dev =
// flagged items.
void scan_flags_list(const uint32_t* word, int64_t n, uint32_t* pos, uint32_t* list,
                     int64_t list_cap, uint32_t* total_dev, uint32_t* status, cudaStream_t s);
// Exclusive scan of uint32 counts into int64 offsets.
void exclusive_scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                               cudaStream_t s);

// ---- stable LSD radix sort (radix_sort.cu) ----
// Sorts (keys, vals) by the low `key_bits` bits of keys, stably. The result
// ends in keys/vals; tmp_keys/tmp_vals are scratch of the same size.
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tmp_keys, uint32_t* tmp_vals,
                      int64_t n, int key_bits, cudaStream_t s);

// Status word written by kernels (bit flags).
enum : uint32_t {
    ST_BAD_INDEX = 1u,
    ST_NONFINITE = 2u,
    ST_BAD_RADIUS = 4u,
    ST_CAPACITY = 8u,
    ST_TIMEOUT = 16u,
};

}  // namespace csl
