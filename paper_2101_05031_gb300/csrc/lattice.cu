// Lattice preparation (Sec. 4): validate the input, order each edge so that
// v_s^z <= v_e^z (Eq. 8), sort the edges by v_s^z and build 32-byte records.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <queue>
#include <vector>

#include "lattice.cuh"

namespace csl {
namespace {

__device__ __forceinline__ uint32_t ord_enc(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float ord_dec(uint32_t u) {
    uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

struct ScanOut {
    uint32_t status;
    uint32_t lo[3], hi[3];
    uint32_t max_r;
    uint32_t max_dz;
};

// Box of the nodes, largest radius and input checks. Each thread keeps its
// own minima and maxima over its grid-stride items; a warp reduces them and
// one lane applies them (a few atomics per warp instead of one per item).
__global__ void k_scan_inputs(const float* __restrict__ nodes, int64_t n_nodes,
                              const int32_t* __restrict__ edges, const float* __restrict__ radius,
                              int64_t n_edges, ScanOut* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t st = 0;
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u}, mr = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += stride) {
        for (int k = 0; k < 3; ++k) {
            float v = nodes[3 * i + k];
            if (!isfinite(v)) { st |= ST_NONFINITE; continue; }
            lo[k] = min(lo[k], ord_enc(v));
            hi[k] = max(hi[k], ord_enc(v));
        }
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_edges; j += stride) {
        int32_t a = edges[2 * j], b = edges[2 * j + 1];
        if (a < 0 || b < 0 || a >= n_nodes || b >= n_nodes) st |= ST_BAD_INDEX;
        float r = radius[j];
        if (!isfinite(r)) st |= ST_NONFINITE;
        else if (!(r > 0.0f)) st |= ST_BAD_RADIUS;
        else mr = max(mr, ord_enc(r));
    }
    const unsigned all = 0xffffffffu;
    for (int k = 0; k < 3; ++k) {
        lo[k] = __reduce_min_sync(all, lo[k]);
        hi[k] = __reduce_max_sync(all, hi[k]);
    }
    mr = __reduce_max_sync(all, mr);
    st = __reduce_or_sync(all, st);
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            if (lo[k] != 0xffffffffu) atomicMin(&out->lo[k], lo[k]);
            if (hi[k] != 0u) atomicMax(&out->hi[k], hi[k]);
        }
        if (mr) atomicMax(&out->max_r, mr);
        if (st) atomicOr(&out->status, st);
    }
}

__global__ void k_prep_keys(const float* __restrict__ nodes, const int32_t* __restrict__ edges,
                            int64_t n_edges, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_edges; j += stride) {
        float za = nodes[3 * (int64_t)edges[2 * j] + 2];
        float zb = nodes[3 * (int64_t)edges[2 * j + 1] + 2];
        keys[j] = ord_enc(zb < za ? zb : za);
        vals[j] = (uint32_t)j;
    }
}

__global__ void k_build_records(const float* __restrict__ nodes, const int32_t* __restrict__ edges,
                                const float* __restrict__ radius, const uint32_t* __restrict__ order,
                                int64_t n_edges, double R, double C, int mode,
                                csl_rec* __restrict__ rec, float4* __restrict__ bxy,
                                float* __restrict__ zlo,
                                float* __restrict__ zhi, uint32_t* __restrict__ sid,
                                ScanOut* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t local_max_dz = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_edges; k += stride) {
        uint32_t j = order[k];
        const float* pa = nodes + 3 * (int64_t)edges[2 * (int64_t)j];
        const float* pb = nodes + 3 * (int64_t)edges[2 * (int64_t)j + 1];
        bool swap = pb[2] < pa[2];
        const float* lo = swap ? pb : pa;
        const float* hi = swap ? pa : pb;
        double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
        double L = sqrt(dx * dx + dy * dy + dz * dz);
        double inv = L > 0.0 ? 1.0 / L : 0.0;
        double rho = radius[j];
        double w;
        if (mode == CSL_MODE_RAW) {
            w = rho;
        } else {
            double q = R * R - rho * rho;
            w = C * 15.0 * (R * R) * (R * R) / (16.0 * q * q * sqrt(q));
        }
        csl_rec r;
        r.ax = lo[0];
        r.ay = lo[1];
        r.az = lo[2];
        r.ux = (float)(dx * inv);
        r.uy = (float)(dy * inv);
        r.uz = (float)(dz * inv);
        r.len = (float)L;
        r.w = (float)w;
        rec[k] = r;
        bxy[k] = make_float4(lo[0], lo[1], hi[0], hi[1]);
        zlo[k] = lo[2];
        zhi[k] = hi[2];
        sid[k] = j | (swap ? 0x80000000u : 0u);
        uint32_t e = ord_enc(__double2float_ru(dz));
        local_max_dz = e > local_max_dz ? e : local_max_dz;
    }
    if (local_max_dz) atomicMax(&out->max_dz, local_max_dz);
}

// The order key of a record: its lower z, bit-encoded so that unsigned order
// is numeric order (the key the device sort uses).
inline uint32_t ord_enc_host(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

}  // namespace

void prepare_lattice_streamed(csl_lattice* L, const int32_t* edges, const float* radius,
                              int64_t batch, cudaStream_t s) {
    const int64_t ne = L->n_edges, nn = L->n_nodes;
    // nodes: the device scan (box, finiteness); edges and radii: on the host
    DevBuf scan_out(sizeof(ScanOut), s);
    ScanOut init;
    init.status = 0;
    for (int k = 0; k < 3; ++k) { init.lo[k] = 0xffffffffu; init.hi[k] = 0u; }
    init.max_r = 0;
    init.max_dz = 0;
    CSL_CUDA(cudaMemcpyAsync(scan_out.get(), &init, sizeof(init), cudaMemcpyHostToDevice, s));
    if (nn > 0) {
        k_scan_inputs<<<grid_for(nn, 256), 256, 0, s>>>(L->nodes.as<float>(), nn, nullptr, nullptr,
                                                        0, scan_out.as<ScanOut>());
        CSL_LAUNCH_CHECK("scan nodes");
    }
    ScanOut h;
    read_to_host(&h, scan_out.get(), sizeof(h), s);
    if (h.status & ST_NONFINITE) fail(CSL_ERR_INVALID_ARG, "non-finite node coordinate or radius");
    float max_r = 0.0f;
    for (int64_t j = 0; j < ne; ++j) {
        const int32_t a = edges[2 * j], b = edges[2 * j + 1];
        if (a < 0 || b < 0 || a >= nn || b >= nn) fail(CSL_ERR_INVALID_ARG, "edge index outside [0, n_nodes)");
        const float r = radius[j];
        if (!isfinite(r)) fail(CSL_ERR_INVALID_ARG, "non-finite node coordinate or radius");
        if (!(r > 0.0f)) fail(CSL_ERR_INVALID_ARG, "radius must be > 0");
        max_r = std::max(max_r, r);
    }
    if (nn > 0)
        for (int k = 0; k < 3; ++k) { L->bbox_lo[k] = ord_dec(h.lo[k]); L->bbox_hi[k] = ord_dec(h.hi[k]); }
    L->max_radius = max_r;
    if (!(L->R > 0.0)) L->R = 1.5 * (double)L->max_radius;
    if (!(L->R > 0.0)) L->R = 1.0;
    if (L->mode == CSL_MODE_PHYSICAL && ne > 0 && !((double)L->max_radius < L->R))
        fail(CSL_ERR_INVALID_ARG, "PHYSICAL mode needs every radius < R");
    L->max_dz = 0;
    L->host_resident = true;
    auto host = [&](size_t bytes) {
        void* p = host_block_alloc(bytes ? bytes : 16);
        if (!p) fail(CSL_ERR_OOM, "host memory for the records");
        return p;
    };
    L->h_rec = (csl_rec*)host((size_t)ne * sizeof(csl_rec));
    L->h_bxy = (float4*)host((size_t)ne * sizeof(float4));
    L->h_zlo = (float*)host((size_t)ne * 4);
    L->h_zhi = (float*)host((size_t)ne * 4);
    L->h_sid = (uint32_t*)host((size_t)ne * 4);
    if (ne == 0) return;
    // every batch: keys, stable sort, records, back to the host as one sorted run
    const int64_t B = std::max<int64_t>(1, std::min(batch, ne));
    std::vector<csl_rec> r_rec(ne);
    std::vector<float4> r_bxy(ne);
    std::vector<float> r_zlo(ne), r_zhi(ne);
    std::vector<uint32_t> r_sid(ne);
    std::vector<int64_t> run_beg;
    {
        DevBuf d_e((size_t)B * 8, s), d_r((size_t)B * 4, s), keys((size_t)B * 4, s),
            vals((size_t)B * 4, s), tk((size_t)B * 4, s), tv((size_t)B * 4, s);
        DevBuf d_rec((size_t)B * sizeof(csl_rec), s), d_bxy((size_t)B * 16, s), d_zlo((size_t)B * 4, s),
            d_zhi((size_t)B * 4, s), d_sid((size_t)B * 4, s);
        for (int64_t b0 = 0; b0 < ne; b0 += B) {
            const int64_t nb = std::min(B, ne - b0);
            run_beg.push_back(b0);
            CSL_CUDA(cudaMemcpyAsync(d_e.get(), edges + 2 * b0, (size_t)nb * 8, cudaMemcpyHostToDevice, s));
            CSL_CUDA(cudaMemcpyAsync(d_r.get(), radius + b0, (size_t)nb * 4, cudaMemcpyHostToDevice, s));
            k_prep_keys<<<grid_for(nb, 256), 256, 0, s>>>(L->nodes.as<float>(), d_e.as<int32_t>(), nb,
                                                         keys.as<uint32_t>(), vals.as<uint32_t>());
            CSL_LAUNCH_CHECK("prep keys (batch)");
            radix_sort_pairs(keys.as<uint32_t>(), vals.as<uint32_t>(), tk.as<uint32_t>(),
                             tv.as<uint32_t>(), nb, 32, s);
            k_build_records<<<grid_for(nb, 256), 256, 0, s>>>(
                L->nodes.as<float>(), d_e.as<int32_t>(), d_r.as<float>(), vals.as<uint32_t>(), nb,
                L->R, L->C, L->mode, d_rec.as<csl_rec>(), d_bxy.as<float4>(), d_zlo.as<float>(),
                d_zhi.as<float>(), d_sid.as<uint32_t>(), scan_out.as<ScanOut>());
            CSL_LAUNCH_CHECK("build records (batch)");
            read_to_host(r_rec.data() + b0, d_rec.get(), (size_t)nb * sizeof(csl_rec), s);
            read_to_host(r_bxy.data() + b0, d_bxy.get(), (size_t)nb * 16, s);
            read_to_host(r_zlo.data() + b0, d_zlo.get(), (size_t)nb * 4, s);
            read_to_host(r_zhi.data() + b0, d_zhi.get(), (size_t)nb * 4, s);
            read_to_host(r_sid.data() + b0, d_sid.get(), (size_t)nb * 4, s);
            for (int64_t k = b0; k < b0 + nb; ++k)   // batch-local edge ids to global ones
                r_sid[k] = ((r_sid[k] & 0x7fffffffu) + (uint32_t)b0) | (r_sid[k] & 0x80000000u);
        }
    }
    read_to_host(&h, scan_out.get(), sizeof(h), s);
    L->max_dz = h.max_dz ? ord_dec(h.max_dz) : 0.0f;
    run_beg.push_back(ne);
    // merge the runs by (key, edge id): the order of one stable sort by key
    struct Head {
        uint64_t key;   // z key << 32 | edge id (unique)
        int run;
        int64_t pos;
    };
    auto cmp = [](const Head& a, const Head& b) { return a.key > b.key; };
    std::priority_queue<Head, std::vector<Head>, decltype(cmp)> heap(cmp);
    auto head_key = [&](int64_t k) {
        return ((uint64_t)ord_enc_host(r_zlo[k]) << 32) | (uint64_t)(r_sid[k] & 0x7fffffffu);
    };
    const int n_runs = (int)run_beg.size() - 1;
    for (int r = 0; r < n_runs; ++r)
        if (run_beg[r] < run_beg[r + 1]) heap.push({head_key(run_beg[r]), r, run_beg[r]});
    int64_t out = 0;
    while (!heap.empty()) {
        const Head t = heap.top();
        heap.pop();
        const int64_t k = t.pos;
        L->h_rec[out] = r_rec[k];
        L->h_bxy[out] = r_bxy[k];
        L->h_zlo[out] = r_zlo[k];
        L->h_zhi[out] = r_zhi[k];
        L->h_sid[out] = r_sid[k];
        ++out;
        if (k + 1 < run_beg[t.run + 1]) heap.push({head_key(k + 1), t.run, k + 1});
    }
}

void prepare_lattice(csl_lattice* L, bool recompute_R, cudaStream_t s) {
    const int64_t ne = L->n_edges, nn = L->n_nodes;
    DevBuf scan_out(sizeof(ScanOut), s);
    ScanOut init;
    init.status = 0;
    for (int k = 0; k < 3; ++k) { init.lo[k] = 0xffffffffu; init.hi[k] = 0u; }
    init.max_r = 0;
    init.max_dz = 0;
    CSL_CUDA(cudaMemcpyAsync(scan_out.get(), &init, sizeof(init), cudaMemcpyHostToDevice, s));
    int64_t nmax = nn > ne ? nn : ne;
    if (nmax > 0) {
        k_scan_inputs<<<grid_for(nmax, 256), 256, 0, s>>>(
            L->nodes.as<float>(), nn, L->edges.as<int32_t>(), L->radius.as<float>(), ne,
            scan_out.as<ScanOut>());
        CSL_LAUNCH_CHECK("scan inputs");
    }
    ScanOut h;
    read_to_host(&h, scan_out.get(), sizeof(h), s);
    if (h.status & ST_BAD_INDEX) fail(CSL_ERR_INVALID_ARG, "edge index outside [0, n_nodes)");
    if (h.status & ST_NONFINITE) fail(CSL_ERR_INVALID_ARG, "non-finite node coordinate or radius");
    if (h.status & ST_BAD_RADIUS) fail(CSL_ERR_INVALID_ARG, "radius must be > 0");
    if (nn > 0)
        for (int k = 0; k < 3; ++k) { L->bbox_lo[k] = ord_dec(h.lo[k]); L->bbox_hi[k] = ord_dec(h.hi[k]); }
    L->max_radius = ne > 0 ? ord_dec(h.max_r) : 0.0f;
    if (recompute_R) {
        if (!(L->R > 0.0)) L->R = 1.5 * (double)L->max_radius;
        if (!(L->R > 0.0)) L->R = 1.0;   // empty lattice: any positive support
    }
    if (L->mode == CSL_MODE_PHYSICAL && ne > 0 && !((double)L->max_radius < L->R))
        fail(CSL_ERR_INVALID_ARG, "PHYSICAL mode needs every radius < R");

    L->rec.ensure_persistent((size_t)(ne > 0 ? ne : 1) * sizeof(csl_rec));
    L->bxy.ensure_persistent((size_t)(ne > 0 ? ne : 1) * sizeof(float4));
    L->zlo.ensure_persistent((size_t)(ne > 0 ? ne : 1) * sizeof(float));
    L->zhi.ensure_persistent((size_t)(ne > 0 ? ne : 1) * sizeof(float));
    L->sid.ensure_persistent((size_t)(ne > 0 ? ne : 1) * sizeof(uint32_t));
    L->max_dz = 0;
    if (ne == 0) return;
    DevBuf keys(ne * 4, s), vals(ne * 4, s), tk(ne * 4, s), tv(ne * 4, s);
    k_prep_keys<<<grid_for(ne, 256), 256, 0, s>>>(L->nodes.as<float>(), L->edges.as<int32_t>(), ne,
                                                 keys.as<uint32_t>(), vals.as<uint32_t>());
    CSL_LAUNCH_CHECK("prep keys");
    radix_sort_pairs(keys.as<uint32_t>(), vals.as<uint32_t>(), tk.as<uint32_t>(),
                     tv.as<uint32_t>(), ne, 32, s);
    k_build_records<<<grid_for(ne, 256), 256, 0, s>>>(
        L->nodes.as<float>(), L->edges.as<int32_t>(), L->radius.as<float>(), vals.as<uint32_t>(),
        ne, L->R, L->C, L->mode, L->rec.as<csl_rec>(), L->bxy.as<float4>(), L->zlo.as<float>(),
        L->zhi.as<float>(),
        L->sid.as<uint32_t>(), scan_out.as<ScanOut>());
    CSL_LAUNCH_CHECK("build records");
    read_to_host(&h, scan_out.get(), sizeof(h), s);
    L->max_dz = h.max_dz ? ord_dec(h.max_dz) : 0.0f;
    L->node_csr_off.release();
    L->node_csr.release();
}

}  // namespace csl
