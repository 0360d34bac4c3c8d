// A device array that grows in place: a range of virtual addresses is
// reserved once and physical memory is mapped behind it, unit by unit, as the
// array grows, so a result assembled chunk by chunk is written where it ends
// up (no gather copy at the end, no second copy of it held meanwhile). The
// driver's virtual memory calls are fetched at run time (types only from
// cuda.h).
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "common.cuh"

namespace csl {
namespace {

struct Vmm {
    CUresult (*reserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
    CUresult (*addr_free)(CUdeviceptr, size_t) = nullptr;
    CUresult (*create)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*,
                       unsigned long long) = nullptr;
    CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
    CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle,
                    unsigned long long) = nullptr;
    CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
    CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t) = nullptr;
    CUresult (*granularity)(size_t*, const CUmemAllocationProp*,
                            CUmemAllocationGranularity_flags) = nullptr;
    bool ok = false;
};

template <class F>
bool entry(const char* name, F& f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return false;
    }
    f = reinterpret_cast<F>(p);
    return true;
}

const Vmm& vmm() {
    static Vmm v = [] {
        Vmm r;
        r.ok = entry("cuMemAddressReserve", r.reserve) && entry("cuMemAddressFree", r.addr_free) &&
               entry("cuMemCreate", r.create) && entry("cuMemRelease", r.release) &&
               entry("cuMemMap", r.map) && entry("cuMemUnmap", r.unmap) &&
               entry("cuMemSetAccess", r.set_access) &&
               entry("cuMemGetAllocationGranularity", r.granularity);
        return r;
    }();
    return v;
}

CUmemAllocationProp device_prop(int dev) {
    CUmemAllocationProp prop = {};
    prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    prop.location.id = dev;
    return prop;
}

void vmm_check(CUresult r, const char* what) {
    if (r == CUDA_SUCCESS) return;
    if (r == CUDA_ERROR_OUT_OF_MEMORY) fail(CSL_ERR_OOM, std::string(what) + ": out of memory");
    fail(CSL_ERR_CUDA, std::string(what) + " failed (driver error " + std::to_string((int)r) + ")");
}

// Physical memory is mapped in units of about 512 MiB; a freed array's units
// go back to a per-process cache (up to 64 GiB, as the page-locked host
// blocks), from which the next array maps them again without allocating.
std::mutex g_unit_mu;
std::vector<std::pair<unsigned long long, int>>& unit_cache() {   // (handle, device)
    static std::vector<std::pair<unsigned long long, int>> c;
    return c;
}
constexpr size_t kUnitTarget = (size_t)512 << 20;
constexpr size_t kUnitCacheBytes = (size_t)64 << 30;

size_t unit_bytes(size_t gran) { return (size_t)ceil_div((int64_t)kUnitTarget, (int64_t)gran) * gran; }

// Arrays handed to callers (csl_contours), by base address.
std::mutex g_reg_mu;
std::unordered_map<void*, GrowMap*>& registry() {
    static std::unordered_map<void*, GrowMap*> r;
    return r;
}

}  // namespace

bool growmap_available() { return vmm().ok; }

void GrowMap::reserve(size_t bytes) {
    const Vmm& v = vmm();
    if (!v.ok) fail(CSL_ERR_CUDA, "the driver's virtual memory calls are not available");
    CSL_CUDA(cudaGetDevice(&dev_));
    const CUmemAllocationProp prop = device_prop(dev_);
    vmm_check(v.granularity(&gran_, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED), "granularity");
    if (gran_ == 0) gran_ = (size_t)2 << 20;
    const size_t unit = unit_bytes(gran_);
    reserved_ = std::max<size_t>(ceil_div((int64_t)bytes, (int64_t)unit) * unit, unit);
    vmm_check(v.reserve(&va_, reserved_, 0, 0, 0), "address reservation");
}

void GrowMap::ensure(size_t bytes) {
    if (bytes <= mapped_) return;
    if (bytes > reserved_) fail(CSL_ERR_CAPACITY, "a growing result exceeds its address range");
    const Vmm& v = vmm();
    const size_t unit = unit_bytes(gran_);
    const size_t from = mapped_;
    while (mapped_ < bytes) {
        if (mapped_ + unit > reserved_) fail(CSL_ERR_CAPACITY, "a growing result exceeds its address range");
        unsigned long long h = 0;
        {
            std::lock_guard<std::mutex> lk(g_unit_mu);
            auto& c = unit_cache();
            for (size_t i = c.size(); i-- > 0;)
                if (c[i].second == dev_) {
                    h = c[i].first;
                    c.erase(c.begin() + (std::ptrdiff_t)i);
                    break;
                }
        }
        if (!h) {
            const CUmemAllocationProp prop = device_prop(dev_);
            CUmemGenericAllocationHandle nh;
            vmm_check(v.create(&nh, unit, &prop, 0), "physical allocation");
            h = (unsigned long long)nh;
        }
        const CUresult r = v.map(va_ + mapped_, unit, 0, (CUmemGenericAllocationHandle)h, 0);
        if (r != CUDA_SUCCESS) {
            v.release((CUmemGenericAllocationHandle)h);
            vmm_check(r, "mapping");
        }
        handles_.push_back({h, unit});
        mapped_ += unit;
    }
    CUmemAccessDesc acc = {};
    acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    acc.location.id = dev_;
    acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    vmm_check(v.set_access(va_ + from, mapped_ - from, &acc, 1), "access");
}

void GrowMap::free_all() {
    if (!va_) return;
    const Vmm& v = vmm();
    cudaDeviceSynchronize();   // no kernel may still use the memory
    size_t off = 0;
    for (const auto& hp : handles_) {
        v.unmap(va_ + off, hp.second);
        off += hp.second;
        std::lock_guard<std::mutex> lk(g_unit_mu);
        auto& c = unit_cache();
        if ((c.size() + 1) * hp.second <= kUnitCacheBytes) c.push_back({hp.first, dev_});
        else v.release((CUmemGenericAllocationHandle)hp.first);
    }
    handles_.clear();
    v.addr_free(va_, reserved_);
    va_ = 0;
    reserved_ = mapped_ = 0;
}

GrowMap::~GrowMap() { free_all(); }

void* GrowMap::hand_over() {
    void* p = base();
    if (!p) return nullptr;
    GrowMap* g = new GrowMap();
    std::swap(g->va_, va_);
    std::swap(g->reserved_, reserved_);
    std::swap(g->mapped_, mapped_);
    std::swap(g->gran_, gran_);
    std::swap(g->dev_, dev_);
    std::swap(g->handles_, handles_);
    std::lock_guard<std::mutex> lk(g_reg_mu);
    registry()[p] = g;
    return p;
}

bool growmap_free(void* p) {
    if (!p) return false;
    GrowMap* g = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        auto it = registry().find(p);
        if (it == registry().end()) return false;
        g = it->second;
        registry().erase(it);
    }
    delete g;
    return true;
}

}  // namespace csl
