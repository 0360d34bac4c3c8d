// Topology-preserving simplification of marching-squares contours (the paper
// smooths and simplifies its marching-squares boundaries without creating
// intersections before writing tool paths, Sec. 4).
//
// Every contour vertex lies on a grid edge e and its loop runs from the cell
// on one side of e into the cell on the other. A vertex (loop position q, the
// loop's head at q = 0) is dropped when q is odd in a loop of at least 5
// vertices (its neighbours stay, the loop keeps at least 3), neither cell
// beside e carries a crossing on an edge other than the loop's own two (so
// both cells hold only this loop's segments, and the convex 1 x 2 block they
// form contains the new chord and no other contour piece), and the vertex
// lies within `tol` of the line through its neighbours (decided in FP64).
//
// Device work: each loop's layer, a per-layer bitmap of the grid edges that
// carry a crossing, the keep decisions per loop, a scan of the kept counts and
// the compaction.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace csl {
namespace {

struct SpGrid {
    int32_t W, H;          // padded sample grid
    int64_t words;         // bitmap words per layer
};

__global__ void k_sp_loop_layer(const int64_t* __restrict__ layer_off, int n_layers,
                                int64_t n_loops, int32_t* __restrict__ loop_layer) {
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < n_loops;
         L += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_layers;   // last layer whose first loop is <= L
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (layer_off[mid] <= L) lo = mid; else hi = mid;
        }
        loop_layer[L] = lo;
    }
}

// An edge id outside the padded grid (contours of another grid) is skipped
// and reported through *bad.
__global__ void k_sp_mark(const int64_t* __restrict__ loop_off, const int32_t* __restrict__ eid,
                          const int32_t* __restrict__ loop_layer, int64_t n_loops, SpGrid g,
                          uint32_t* __restrict__ bits, uint32_t* bad) {
    const int64_t n_ids = 2 * (int64_t)g.W * g.H;
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < n_loops;
         L += (int64_t)gridDim.x * blockDim.x) {
        uint32_t* row = bits + (int64_t)loop_layer[L] * g.words;
        for (int64_t v = loop_off[L]; v < loop_off[L + 1]; ++v) {
            const int64_t e = eid[v];
            if (e < 0 || e >= n_ids) {
                atomicOr(bad, 1u);
                continue;
            }
            atomicOr(row + (e >> 5), 1u << (uint32_t)(e & 31));
        }
    }
}

__device__ __forceinline__ bool has_edge(const uint32_t* row, int64_t e, const SpGrid& g) {
    if (e < 0 || (e >> 5) >= g.words) return false;
    return (row[e >> 5] >> (e & 31)) & 1u;
}

// Whether cell (I, J) has a crossing on an edge other than the loop's own
// edges a, b, c (its predecessor's, its own and its successor's).
__device__ __forceinline__ bool other_crossing(int I, int J, int64_t a, int64_t b, int64_t c,
                                               const uint32_t* row, const SpGrid& g) {
    if (I < 0 || J < 0 || I > g.W - 2 || J > g.H - 2) return false;
    const int64_t e[4] = {2 * ((int64_t)J * g.W + I), 2 * ((int64_t)(J + 1) * g.W + I),
                          2 * ((int64_t)J * g.W + I) + 1, 2 * ((int64_t)J * g.W + I + 1) + 1};
    for (int k = 0; k < 4; ++k)
        if (e[k] != a && e[k] != b && e[k] != c && has_edge(row, e[k], g)) return true;
    return false;
}

__global__ void k_sp_keep(const int64_t* __restrict__ loop_off, const int32_t* __restrict__ eid,
                          const float* __restrict__ xy, const int32_t* __restrict__ loop_layer,
                          int64_t n_loops, SpGrid g, const uint32_t* __restrict__ bits, double tol,
                          uint8_t* __restrict__ keep, uint32_t* __restrict__ kept) {
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < n_loops;
         L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = loop_off[L], b = loop_off[L + 1], n = b - a;
        const uint32_t* row = bits + (int64_t)loop_layer[L] * g.words;
        int64_t count = n;
        for (int64_t v = a; v < b; ++v) keep[v] = 1;
        if (n >= 5) {
            for (int64_t q = 1; q < n; q += 2) {
                const int64_t v = a + q, p = a + q - 1, s = a + (q + 1) % n;
                const int64_t ev = eid[v], ep = eid[p], es = eid[s];
                // the two cells beside edge ev
                // a valid ev is below 2 W H < 2^31: a 32-bit division (an
                // invalid one is reported by k_sp_mark; the cell lookups below
                // bound-check whatever I, J it gives)
                const uint32_t base = (uint32_t)ev >> 1;
                const int J = (int)(base / (uint32_t)g.W),
                          I = (int)(base - (uint32_t)J * (uint32_t)g.W);
                int I0, J0;
                if (ev & 1) {
                    I0 = I - 1;
                    J0 = J;
                } else {
                    I0 = I;
                    J0 = J - 1;
                }
                if (other_crossing(I0, J0, ep, ev, es, row, g) ||
                    other_crossing(I, J, ep, ev, es, row, g))
                    continue;
                const double px = xy[2 * p], py = xy[2 * p + 1];
                const double sx = xy[2 * s], sy = xy[2 * s + 1];
                const double vx = xy[2 * v], vy = xy[2 * v + 1];
                const double dx = sx - px, dy = sy - py;
                const double L2 = dx * dx + dy * dy;
                if (L2 == 0.0) continue;
                const double cross = (vx - px) * dy - (vy - py) * dx;
                if (fabs(cross) <= tol * sqrt(L2)) {
                    keep[v] = 0;
                    --count;
                }
            }
        }
        kept[L] = (uint32_t)count;
    }
}

__global__ void k_sp_write(const int64_t* __restrict__ loop_off, const int32_t* __restrict__ eid,
                           const float* __restrict__ xy, const uint8_t* __restrict__ keep,
                           const int64_t* __restrict__ new_off, int64_t n_loops,
                           int32_t* __restrict__ oeid, float* __restrict__ oxy) {
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < n_loops;
         L += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = new_off[L];
        for (int64_t v = loop_off[L]; v < loop_off[L + 1]; ++v)
            if (keep[v]) {
                oeid[o] = eid[v];
                oxy[2 * o] = xy[2 * v];
                oxy[2 * o + 1] = xy[2 * v + 1];
                ++o;
            }
    }
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_simplify_contours(const csl_contours* in, int32_t nx, int32_t ny,
                                            double tol, void* stream, csl_contours** out) {
    csl_contours* c = nullptr;
    try {
        if (!in || !out) fail(CSL_ERR_INVALID_ARG, "NULL argument");
        *out = nullptr;
        if (!in->on_device) fail(CSL_ERR_INVALID_ARG, "contours must be on the device");
        if (!in->edge_id) fail(CSL_ERR_INVALID_ARG, "contours need their edge ids");
        if (nx < 1 || ny < 1 || nx > 32000 || ny > 32000)
            fail(CSL_ERR_INVALID_ARG, "nx, ny must be in [1, 32000]");
        if (!(tol >= 0.0) || !isfinite(tol)) fail(CSL_ERR_INVALID_ARG, "tol must be >= 0");
        cudaStream_t s = (cudaStream_t)stream;
        SpGrid g;
        g.W = nx + 2;
        g.H = ny + 2;
        g.words = ceil_div(2 * (int64_t)g.W * g.H, 32);
        const int n_layers = in->n_layers;
        const int64_t n_loops = in->n_loops, n_verts = in->n_verts;
        if ((double)n_layers * (double)g.words * 4.0 > (double)(16ll << 30))
            fail(CSL_ERR_CAPACITY, "edge bitmap above 16 GiB: simplify fewer layers at a time");
        c = new csl_contours();
        c->n_layers = n_layers;
        c->on_device = 1;
        c->n_loops = n_loops;
        auto dst_alloc = [&](void** p, size_t bytes) {
            if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
                cudaGetLastError();
                fail(CSL_ERR_OOM, "device allocation of the contours failed");
            }
        };
        dst_alloc((void**)&c->layer_loop_off, (size_t)(n_layers + 1) * 8);
        dst_alloc((void**)&c->loop_vert_off, (size_t)(n_loops + 1) * 8);
        CSL_CUDA(cudaMemcpyAsync(c->layer_loop_off, in->layer_loop_off, (size_t)(n_layers + 1) * 8,
                                 cudaMemcpyDeviceToDevice, s));
        DevBuf d_layer((size_t)std::max<int64_t>(n_loops, 1) * 4, s);
        DevBuf d_bits((size_t)std::max<int64_t>((int64_t)n_layers * g.words, 1) * 4, s);
        DevBuf d_keep((size_t)std::max<int64_t>(n_verts, 1), s);
        DevBuf d_kept((size_t)std::max<int64_t>(n_loops, 1) * 4, s);
        DevBuf d_tot(8, s), d_bad(4, s);
        int64_t n_out = 0;
        if (n_loops > 0) {
            CSL_CUDA(cudaMemsetAsync(d_bad.get(), 0, 4, s));
            CSL_CUDA(cudaMemsetAsync(d_bits.get(), 0, (size_t)n_layers * g.words * 4, s));
            k_sp_loop_layer<<<grid_for(n_loops, 256), 256, 0, s>>>(in->layer_loop_off, n_layers,
                                                                   n_loops, d_layer.as<int32_t>());
            CSL_LAUNCH_CHECK("simplify loop layers");
            k_sp_mark<<<grid_for(n_loops, 256), 256, 0, s>>>(in->loop_vert_off, in->edge_id,
                                                             d_layer.as<int32_t>(), n_loops, g,
                                                             d_bits.as<uint32_t>(),
                                                             d_bad.as<uint32_t>());
            CSL_LAUNCH_CHECK("simplify edge bitmap");
            k_sp_keep<<<grid_for(n_loops, 256), 256, 0, s>>>(
                in->loop_vert_off, in->edge_id, in->xy, d_layer.as<int32_t>(), n_loops, g,
                d_bits.as<uint32_t>(), tol, d_keep.as<uint8_t>(), d_kept.as<uint32_t>());
            CSL_LAUNCH_CHECK("simplify decisions");
            exclusive_scan_u32_to_i64(d_kept.as<uint32_t>(), c->loop_vert_off, n_loops,
                                      d_tot.as<int64_t>(), s);
            n_out = read_i64(d_tot.as<int64_t>(), s);
            uint32_t bad = 0;
            read_to_host(&bad, d_bad.get(), 4, s);
            if (bad) fail(CSL_ERR_INVALID_ARG, "edge ids outside the nx x ny grid");
            CSL_CUDA(cudaMemcpyAsync(c->loop_vert_off + n_loops, d_tot.get(), 8,
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            CSL_CUDA(cudaMemsetAsync(c->loop_vert_off, 0, 8, s));
        }
        c->n_verts = n_out;
        dst_alloc((void**)&c->xy, (size_t)n_out * 8);
        dst_alloc((void**)&c->edge_id, (size_t)n_out * 4);
        if (n_loops > 0) {
            k_sp_write<<<grid_for(n_loops, 256), 256, 0, s>>>(
                in->loop_vert_off, in->edge_id, in->xy, d_keep.as<uint8_t>(), c->loop_vert_off,
                n_loops, c->edge_id, c->xy);
            CSL_LAUNCH_CHECK("simplify write");
        }
        CSL_CUDA(cudaStreamSynchronize(s));
        *out = c;
        return CSL_OK;
    } catch (const Error& e) {
        if (c) csl_contours_free(c);
        set_last_error(e.what());
        return e.code;
    } catch (...) {
        if (c) csl_contours_free(c);
        set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}
