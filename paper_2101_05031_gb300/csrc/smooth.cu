// Topology-preserving smoothing of marching-squares contours (the paper
// smooths its marching-squares boundaries, without creating intersections,
// before it writes tool paths, Sec. 4).
//
// Every contour vertex lies on a grid edge e of the padded sample grid
// (W = nx + 2): horizontal edge 2 (J W + I) from sample (I, J) to (I + 1, J),
// vertical edge 2 (J W + I) + 1 from (I, J) to (I, J + 1); padded sample
// (I, J) sits at (x0 + (I - 1/2) px, y0 + (J - 1/2) px). A vertex moves only
// along its own edge: in each of K Jacobi iterations its free coordinate a
// (x on a horizontal edge, y on a vertical one) becomes a + lam (m - a), m the
// mean of the same coordinate of its loop predecessor and successor, clamped
// to [lo + mu px, lo + (1 - mu) px] (lo: the edge's first sample), in float32
// with every operation rounded on its own, in the order m = 0.5 (a_p + a_s),
// a + lam (m - a), lo = c0 + I px (c0 = x0 - px / 2, or the y and row
// counterparts) and the two bounds, so that results are the same bit for bit
// wherever the same operations run. Loops of fewer than 3 vertices stay as they are. Each
// segment joins vertices on two edges of one cell (or of the 1 x 2 block of a
// vertex that simplification dropped) and every vertex stays strictly inside
// its edge, so every segment stays in its cell; a saddle cell's two segments
// lie strictly on the two sides of a diagonal. No crossing can appear.
//
// Device work: the loop of every vertex, a check of the edge ids against the
// grid, then one launch per iteration (a thread per vertex, two buffers).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace csl {
namespace {

struct SmConst {
    int32_t W;
    int64_t n_ids;        // 2 W H
    float cx0, cy0, px, lam;   // x0 - px / 2, y0 - px / 2 (rounded once from FP64)
    float m_lo, m_hi;          // mu px and (1 - mu) px
};

__global__ void k_sm_loop_of(const int64_t* __restrict__ loop_off, int64_t n_loops,
                             int32_t* __restrict__ vloop) {
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < n_loops;
         L += (int64_t)gridDim.x * blockDim.x)
        for (int64_t v = loop_off[L]; v < loop_off[L + 1]; ++v) vloop[v] = (int32_t)L;
}

__global__ void k_sm_check(const int32_t* __restrict__ eid, int64_t n, int64_t n_ids,
                           uint32_t* bad) {
    bool b = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        b |= eid[v] < 0 || (int64_t)eid[v] >= n_ids;
    if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1u);
}

__global__ void k_sm_step(const int64_t* __restrict__ loop_off, const int32_t* __restrict__ vloop,
                          const int32_t* __restrict__ eid, const float2* __restrict__ src,
                          int64_t n, SmConst g, float2* __restrict__ dst) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        float2 P = src[v];
        const int32_t L = vloop[v];
        const int64_t a = loop_off[L], b = loop_off[L + 1];
        const int64_t e = eid[v];
        if (b - a >= 3 && e >= 0 && e < g.n_ids) {   // the ids were checked before
            const int64_t p = v == a ? b - 1 : v - 1;
            const int64_t s = v == b - 1 ? a : v + 1;
            const float2 Pp = src[p], Ps = src[s];
            // e < 2 W H < 2^31: 32-bit division (a 64-bit one is a long
            // emulated sequence per vertex)
            const uint32_t base = (uint32_t)e >> 1;
            const int J = (int)(base / (uint32_t)g.W), I = (int)(base - (uint32_t)J * (uint32_t)g.W);
            const bool vert = e & 1;   // vertical edge: y moves; horizontal: x moves
            const float lo = __fadd_rn(vert ? g.cy0 : g.cx0,
                                       __fmul_rn((float)(vert ? J : I), g.px));
            const float av = vert ? P.y : P.x;
            const float m = __fmul_rn(0.5f, __fadd_rn(vert ? Pp.y : Pp.x, vert ? Ps.y : Ps.x));
            const float an = __fadd_rn(av, __fmul_rn(g.lam, __fsub_rn(m, av)));
            const float a = fminf(fmaxf(an, __fadd_rn(lo, g.m_lo)), __fadd_rn(lo, g.m_hi));
            if (vert) P.y = a;
            else P.x = a;
        }
        dst[v] = P;
    }
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_smooth_contours(csl_contours* c, double x0, double y0, double pixel,
                                          int32_t nx, int32_t ny, double lambda, double margin,
                                          int32_t iterations, void* stream) {
    try {
        if (!c) fail(CSL_ERR_INVALID_ARG, "NULL argument");
        if (!c->on_device) fail(CSL_ERR_INVALID_ARG, "contours must be on the device");
        if (!c->edge_id) fail(CSL_ERR_INVALID_ARG, "contours need their edge ids");
        if (nx < 1 || ny < 1 || nx > 32000 || ny > 32000)
            fail(CSL_ERR_INVALID_ARG, "nx, ny must be in [1, 32000]");
        if (!isfinite(x0) || !isfinite(y0)) fail(CSL_ERR_INVALID_ARG, "non-finite origin");
        if (!(pixel > 0.0) || !isfinite(pixel)) fail(CSL_ERR_INVALID_ARG, "pixel must be > 0");
        if (!(lambda >= 0.0 && lambda <= 1.0)) fail(CSL_ERR_INVALID_ARG, "lambda in [0, 1]");
        if (!(margin > 0.0 && margin <= 0.5)) fail(CSL_ERR_INVALID_ARG, "margin in (0, 1/2]");
        if (iterations < 0 || iterations > 10000)
            fail(CSL_ERR_INVALID_ARG, "iterations in [0, 10000]");
        if (c->n_loops > 0x7fffffffLL) fail(CSL_ERR_CAPACITY, "more than 2^31 - 1 loops");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n = c->n_verts, n_loops = c->n_loops;
        if (n == 0 || iterations == 0) {
            CSL_CUDA(cudaStreamSynchronize(s));
            return CSL_OK;
        }
        SmConst g;
        g.W = nx + 2;
        g.n_ids = 2 * (int64_t)(nx + 2) * (ny + 2);
        g.cx0 = (float)(x0 - 0.5 * pixel);
        g.cy0 = (float)(y0 - 0.5 * pixel);
        g.px = (float)pixel;
        g.lam = (float)lambda;
        g.m_lo = (float)(margin * pixel);
        g.m_hi = (float)((1.0 - margin) * pixel);
        DevBuf d_bad(4, s), d_vloop((size_t)n * 4, s), d_tmp((size_t)n * 8, s);
        CSL_CUDA(cudaMemsetAsync(d_bad.get(), 0, 4, s));
        k_sm_check<<<grid_for(n, 256), 256, 0, s>>>(c->edge_id, n, g.n_ids, d_bad.as<uint32_t>());
        CSL_LAUNCH_CHECK("smooth edge-id check");
        uint32_t bad = 0;
        read_to_host(&bad, d_bad.get(), 4, s);
        if (bad) fail(CSL_ERR_INVALID_ARG, "edge ids outside the nx x ny grid");
        k_sm_loop_of<<<grid_for(n_loops, 256), 256, 0, s>>>(c->loop_vert_off, n_loops,
                                                             d_vloop.as<int32_t>());
        CSL_LAUNCH_CHECK("smooth vertex loops");
        float2* bufs[2] = {reinterpret_cast<float2*>(c->xy), d_tmp.as<float2>()};
        for (int it = 0; it < iterations; ++it) {
            k_sm_step<<<grid_for(n, 256), 256, 0, s>>>(c->loop_vert_off, d_vloop.as<int32_t>(),
                                                       c->edge_id, bufs[it & 1], n, g,
                                                       bufs[(it + 1) & 1]);
            CSL_LAUNCH_CHECK("smooth step");
        }
        if (iterations & 1)
            CSL_CUDA(cudaMemcpyAsync(c->xy, d_tmp.get(), (size_t)n * 8, cudaMemcpyDeviceToDevice,
                                     s));
        CSL_CUDA(cudaStreamSynchronize(s));
        return CSL_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (...) {
        set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}
