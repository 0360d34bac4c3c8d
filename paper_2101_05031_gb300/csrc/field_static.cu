// csl_field_layers_static: the field on a few layers, for callers that cannot
// allocate device memory. Its only scratch is the fixed array below, which
// every GPU that loads this library holds until the process exits.
//
// Scratch layout: a 256-byte header (word 0: validation status) followed by
// CSL_STATIC_MAX_EDGES prepared edge records of 32 bytes. Calls share the
// array: the status word is cleared at the start of every call, the records
// are rewritten by every call, and two calls whose GPU work overlaps (other
// streams, other host threads) race on it.
#include <cuda.h>   // driver API types only: cuCtxGetCurrent/cuCtxGetId are fetched at run time
#include <math.h>

#include <mutex>

#include "lattice.cuh"

namespace csl {
namespace {

constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)CSL_STATIC_MAX_EDGES * sizeof(csl_rec);
static_assert(sizeof(csl_rec) == 32, "record layout");

__device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of g_static_scratch in the current context. Host code cannot
// use the symbol's name as a device address, so it is looked up with
// cudaGetSymbolAddress once per device, with that device current, and cached.
// With lazy module loading (the CUDA default) that first look-up also loads
// this file's module and so reserves the array; it may allocate and
// synchronise, so make the first call during set-up, before any stream
// capture. The cache is keyed on the context's unique id: after a
// cudaDeviceReset the next call runs in a new primary context, finds a
// different id and looks the address up again instead of using a stale one.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
    });
    if (!get_current || !get_id) fail(CSL_ERR_CUDA, "driver entry points for the context id");
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        fail(CSL_ERR_CUDA, "no current CUDA context");
    return id;
}

void* scratch_address() {
    static std::mutex mu;
    static void* addr[64] = {};
    static unsigned long long ctx_of[64] = {};
    int dev = 0;
    CSL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(CSL_ERR_NOT_READY, "device index out of range");
    CSL_CUDA(cudaSetDevice(dev));   // makes the device's primary context current (no allocation)
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || ctx_of[dev] != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(CSL_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                   cudaGetErrorString(e));
        }
        addr[dev] = p;
        ctx_of[dev] = ctx;
    }
    return addr[dev];
}

// One record per edge, in edge order (no sort): v_s (lower z), unit
// direction, length, weight. Invalid edges are reported and given weight 0.
__global__ void k_static_prep(const float* __restrict__ nodes, int64_t n_nodes,
                              const int32_t* __restrict__ edges, const float* __restrict__ radius,
                              int64_t n_edges, double R, double C, int mode,
                              csl_rec* __restrict__ rec, uint32_t* status) {
    // every node coordinate, as csl_lattice_upload checks, also those no edge uses
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_nodes;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(nodes[i])) atomicOr(status, ST_NONFINITE);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_edges;
         j += (int64_t)gridDim.x * blockDim.x) {
        csl_rec r = {0, 0, 0, 0, 0, 0, 0, 0};
        const int32_t i0 = edges[2 * j], i1 = edges[2 * j + 1];
        const float rho = radius[j];
        uint32_t st = 0;
        if (i0 < 0 || i1 < 0 || i0 >= n_nodes || i1 >= n_nodes) st |= ST_BAD_INDEX;
        if (!isfinite(rho)) st |= ST_NONFINITE;
        else if (!(rho > 0.0f) || (mode == CSL_MODE_PHYSICAL && !((double)rho < R)))
            st |= ST_BAD_RADIUS;
        if (!st) {
            const float* pa = nodes + 3 * (int64_t)i0;
            const float* pb = nodes + 3 * (int64_t)i1;
            if (!isfinite(pa[0]) || !isfinite(pa[1]) || !isfinite(pa[2]) || !isfinite(pb[0]) ||
                !isfinite(pb[1]) || !isfinite(pb[2]))
                st |= ST_NONFINITE;
        }
        if (st) {
            atomicOr(status, st);
            rec[j] = r;
            continue;
        }
        const float* pa = nodes + 3 * (int64_t)i0;
        const float* pb = nodes + 3 * (int64_t)i1;
        const bool swap = pb[2] < pa[2];
        const float* lo = swap ? pb : pa;
        const float* hi = swap ? pa : pb;
        const double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1];
        const double dz = (double)hi[2] - lo[2];
        const double L = sqrt(dx * dx + dy * dy + dz * dz);
        const double inv = L > 0.0 ? 1.0 / L : 0.0;
        double w = rho;
        if (mode != CSL_MODE_RAW) {
            const double q = R * R - (double)rho * rho;
            w = C * 15.0 * (R * R) * (R * R) / (16.0 * q * q * sqrt(q));
        }
        r.ax = lo[0];
        r.ay = lo[1];
        r.az = lo[2];
        r.ux = (float)(dx * inv);
        r.uy = (float)(dy * inv);
        r.uz = (float)(dz * inv);
        r.len = (float)L;
        r.w = (float)w;
        rec[j] = r;
    }
}

struct StaticConst {
    int32_t nx, ny, ntx;
    int32_t n_edges;
    double x0, y0, px, z0, dz;
    float R2, inv_R4, fpx, cull;
};

// One CTA per (16x16-pixel tile, layer). The CTA streams every record
// through shared memory, keeps (in edge order) those whose support can reach
// the tile at this layer, and each thread sums the kept terms for its pixel.
__global__ void __launch_bounds__(256) k_static_field(const csl_rec* __restrict__ rec,
                                                      StaticConst c, float* __restrict__ sigma) {
    __shared__ float4 s_a[256];   // ax, ay, az (tile-local), ux
    __shared__ float4 s_b[256];   // uy, uz, len, w / R^4
    __shared__ uint32_t s_warp[8];
    __shared__ float s_org[6];
    const int tile = blockIdx.x, layer = blockIdx.y;
    const int tx = tile % c.ntx, ty = tile / c.ntx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int il = threadIdx.x & 15, jl = threadIdx.x >> 4;
    if (threadIdx.x == 0) {
        const double ox = c.x0 + (double)(tx * 16) * c.px;
        const double oy = c.y0 + (double)(ty * 16) * c.px;
        const double oz = c.z0 + (double)layer * c.dz;
        s_org[0] = (float)ox;
        s_org[1] = (float)(ox - (double)s_org[0]);
        s_org[2] = (float)oy;
        s_org[3] = (float)(oy - (double)s_org[2]);
        s_org[4] = (float)oz;
        s_org[5] = (float)(oz - (double)s_org[4]);
    }
    __syncthreads();
    const float oxh = s_org[0], oxl = s_org[1], oyh = s_org[2], oyl = s_org[3];
    const float ozh = s_org[4], ozl = s_org[5];
    const float pxl = ((float)il + 0.5f) * c.fpx, pyl = ((float)jl + 0.5f) * c.fpx;
    const float lo_px = 0.5f * c.fpx, hi_px = 15.5f * c.fpx;
    float acc = 0.0f;
    for (int c0 = 0; c0 < c.n_edges; c0 += 256) {
        const int j = c0 + (int)threadIdx.x;
        bool keep = false;
        float4 A = make_float4(0, 0, 0, 0), B = make_float4(0, 0, 0, 0);
        if (j < c.n_edges) {
            const csl_rec r = rec[j];
            const float ax = (r.ax - oxh) - oxl, ay = (r.ay - oyh) - oyl, az = (r.az - ozh) - ozl;
            A = make_float4(ax, ay, az, r.ux);
            B = make_float4(r.uy, r.uz, r.len, r.w * c.inv_R4);
            // the edge clipped to |z| <= cull around this layer, its xy box grown by cull
            float t_lo = 0.0f, t_hi = r.len;
            if (r.uz > 1e-12f) {
                t_lo = fmaxf((-c.cull - az) / r.uz, 0.0f);
                t_hi = fminf((c.cull - az) / r.uz, r.len);
            } else if (fabsf(az) > c.cull) {
                t_lo = 1.0f;
                t_hi = 0.0f;
            }
            if (r.w != 0.0f && t_lo <= t_hi) {
                const float xa = fmaf(t_lo, r.ux, ax), xb = fmaf(t_hi, r.ux, ax);
                const float ya = fmaf(t_lo, r.uy, ay), yb = fmaf(t_hi, r.uy, ay);
                keep = fmaxf(xa, xb) + c.cull >= lo_px && fminf(xa, xb) - c.cull <= hi_px &&
                       fmaxf(ya, yb) + c.cull >= lo_px && fminf(ya, yb) - c.cull <= hi_px;
            }
        }
        // order-preserving compaction of the kept records
        const uint32_t ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[warp] = __popc(ball);
        __syncthreads();
        uint32_t base = 0, total = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t n = s_warp[w];
            if (w < warp) base += n;
            total += n;
        }
        if (keep) {
            const uint32_t pos = base + __popc(ball & ((1u << lane) - 1u));
            s_a[pos] = A;
            s_b[pos] = B;
        }
        __syncthreads();
        for (uint32_t k = 0; k < total; ++k) {
            const float4 a = s_a[k], b = s_b[k];
            const float dx = pxl - a.x, dy = pyl - a.y, dz = -a.z;
            const float t0 = fmaf(dz, b.y, fmaf(dy, b.x, dx * a.w));
            const float ex = fmaf(-t0, a.w, dx), ey = fmaf(-t0, b.x, dy), ez = fmaf(-t0, b.y, dz);
            const float h2 = fmaxf(c.R2 - fmaf(ez, ez, fmaf(ey, ey, ex * ex)), 0.0f);
            const float w = sqrtf(h2);
            const float tau1 = fmaxf(-t0, -w), tau2 = fminf(b.z - t0, w);
            const float d = fmaxf(tau2 - tau1, 0.0f);      // 2 h
            const float s = tau2 + tau1;                    // 2 m
            const float cc = fmaf(-0.25f * s, s, h2);       // w^2 - m^2
            const float dd = 0.15f * d * d;                 // 0.6 h^2
            const float Av = cc - dd;
            const float B2 = dd * s * s;
            const float I = d * fmaf(5.0f / 9.0f, fmaf(Av, Av, B2), (4.0f / 9.0f) * cc * cc);
            acc = fmaf(b.w, I, acc);
        }
        __syncthreads();
    }
    const int gi = tx * 16 + il, gj = ty * 16 + jl;
    if (gi < c.nx && gj < c.ny) sigma[((int64_t)layer * c.ny + gj) * c.nx + gi] = acc;
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_field_layers_static(const float* nodes_xyz, int64_t n_nodes,
                                              const int32_t* edges_ij, const float* radius,
                                              int64_t n_edges, double R, double C, int32_t mode,
                                              const csl_slice_desc* desc, float* sigma_out,
                                              void* stream) {
    try {
        auto require = [](bool ok, const char* msg) {
            if (!ok) fail(CSL_ERR_INVALID_ARG, msg);
        };
        require(desc != nullptr, "desc is NULL");
        require(n_nodes >= 0 && n_edges >= 0, "negative size");
        if (n_edges > CSL_STATIC_MAX_EDGES)
            fail(CSL_ERR_CAPACITY, "n_edges exceeds the static scratch of "
                                   "csl_field_layers_static (at most CSL_STATIC_MAX_EDGES = " +
                                       std::to_string(CSL_STATIC_MAX_EDGES) + " edges)");
        require(n_nodes <= 0x7fffffffLL, "more than 2^31 - 1 nodes");
        require(n_nodes == 0 || nodes_xyz != nullptr, "nodes_xyz is NULL");
        require(n_edges == 0 || (edges_ij != nullptr && radius != nullptr),
                "edges_ij or radius is NULL");
        require(isfinite(R) && R > 0.0, "R must be > 0 (no default here)");
        if (C == 0.0) C = 1.0;
        require(isfinite(C) && C > 0.0, "C must be > 0");
        require(mode == CSL_MODE_PHYSICAL || mode == CSL_MODE_RAW, "unknown mode");
        const csl_slice_desc& d = *desc;
        require(d.n_layers >= 0 && d.n_layers <= 65535, "n_layers must be in [0, 65535]");
        require(d.nx >= 1 && d.ny >= 1 && d.nx <= 32000 && d.ny <= 32000,
                "nx, ny must be in [1, 32000]");
        require(isfinite(d.pixel) && d.pixel > 0, "pixel must be > 0");
        require(isfinite(d.x0) && isfinite(d.y0) && isfinite(d.z0), "non-finite origin");
        require(isfinite(d.dz), "dz must be finite");   // layer k lies at z0 + k dz
        require(d.n_layers <= 1 || d.dz > 0, "dz must be > 0");
        require(d.n_layers == 0 || sigma_out != nullptr, "sigma_out is NULL");
        if (d.n_layers == 0) return CSL_OK;
        cudaStream_t s = (cudaStream_t)stream;
        unsigned char* base = (unsigned char*)scratch_address();
        uint32_t* status = (uint32_t*)base;
        csl_rec* rec = (csl_rec*)(base + kHeaderBytes);
        CSL_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
        if (n_edges > 0 || n_nodes > 0) {
            k_static_prep<<<grid_for(n_edges > 3 * n_nodes ? n_edges : 3 * n_nodes, 256), 256, 0, s>>>(
                nodes_xyz, n_nodes, edges_ij, radius, n_edges, R, C, mode, rec, status);
            CSL_LAUNCH_CHECK("static prep");
        }
        StaticConst c;
        c.nx = d.nx;
        c.ny = d.ny;
        c.ntx = (d.nx + 15) / 16;
        c.n_edges = (int32_t)n_edges;
        c.x0 = d.x0;
        c.y0 = d.y0;
        c.px = d.pixel;
        c.z0 = d.z0;
        c.dz = d.dz;
        c.R2 = (float)(R * R);
        c.inv_R4 = (float)(1.0 / (R * R * R * R));
        c.fpx = (float)d.pixel;
        c.cull = (float)(R * (1.0 + 1e-5) + 1e-6);
        const int nty = (d.ny + 15) / 16;
        dim3 grid((unsigned)(c.ntx * nty), (unsigned)d.n_layers);
        k_static_field<<<grid, 256, 0, s>>>(rec, c, sigma_out);
        CSL_LAUNCH_CHECK("static field");
        uint32_t st = 0;
        CSL_CUDA(cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
        CSL_CUDA(cudaStreamSynchronize(s));
        if (st & ST_BAD_INDEX) fail(CSL_ERR_INVALID_ARG, "edge index outside [0, n_nodes)");
        if (st & ST_NONFINITE) fail(CSL_ERR_INVALID_ARG, "non-finite node coordinate or radius");
        if (st & ST_BAD_RADIUS)
            fail(CSL_ERR_INVALID_ARG, "radius must be > 0 (and < R in PHYSICAL mode)");
        return CSL_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return CSL_ERR_CUDA;
    }
}
