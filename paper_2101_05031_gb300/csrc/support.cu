// Self-support metrics of a lattice (Sec. 5.3, Eq. 11-14): for every edge, the
// angle theta = arccos |u . t_P| between the edge and the printing direction
// (Eq. 11); an edge with theta <= alpha is fully self-supported. The risky
// fraction of a strut's projected facing-down area is g(theta) = sum_i a_i
// theta^i for theta > alpha and 0 otherwise (Eq. 12, the paper's quintic for
// alpha = pi / 4). Gamma (Eq. 13) = sum over unsupported edges of r L g(theta)
// / sum over all edges of r L; Psi (Eq. 14) = sum over supported edges of L /
// sum of L. Sums in double, per block in a fixed tree order, then the blocks in
// order: deterministic.
#include <math.h>

#include "lattice.cuh"
#include "slice.cuh"

namespace csl {
namespace {

constexpr int kThreads = 256;

struct SupportConst {
    double tx, ty, tz;   // printing direction (unit)
    double alpha;
    double a[6];
};

__device__ __forceinline__ void block_sum4(double (&v)[4], double* out) {
    __shared__ double s[4][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) s[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += s[threadIdx.x][w];
        out[threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_support(const float* __restrict__ nodes,
                                                      const int32_t* __restrict__ edges,
                                                      const float* __restrict__ radius,
                                                      int64_t n_edges, SupportConst c,
                                                      double* __restrict__ partial) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // r L g (unsupported), r L, L (supported), L
    const int64_t per = (n_edges + gridDim.x - 1) / gridDim.x;   // contiguous range per block
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(n_edges, lo + per);
    for (int64_t j = lo + threadIdx.x; j < hi; j += kThreads) {
        const int32_t a = edges[2 * j], b = edges[2 * j + 1];
        const double dx = (double)nodes[3 * b] - nodes[3 * a];
        const double dy = (double)nodes[3 * b + 1] - nodes[3 * a + 1];
        const double dz = (double)nodes[3 * b + 2] - nodes[3 * a + 2];
        const double L = sqrt(dx * dx + dy * dy + dz * dz);
        const double r = (double)radius[j];
        double th = 0.0;
        if (L > 0.0) {
            const double cs = fabs((dx * c.tx + dy * c.ty + dz * c.tz) / L);
            th = acos(cs < 1.0 ? cs : 1.0);
        }
        v[1] += r * L;
        v[3] += L;
        if (th <= c.alpha) {
            v[2] += L;
        } else {
            double g = c.a[5];
            for (int i = 4; i >= 0; --i) g = g * th + c.a[i];
            v[0] += r * L * g;
        }
    }
    block_sum4(v, partial + 4 * (int64_t)blockIdx.x);
}

__global__ void k_support_total(const double* __restrict__ partial, int n_blocks,
                                double* __restrict__ out) {
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int b = 0; b < n_blocks; ++b) t += partial[4 * b + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_support_metrics(const csl_lattice* L, const double* t_p, double alpha,
                                          const double* coeffs, double* gamma, double* psi,
                                          void* stream) {
    try {
        if (!L || !t_p || !gamma || !psi) fail(CSL_ERR_INVALID_ARG, "NULL argument");
        require_device_resident(L);
        const double n = sqrt(t_p[0] * t_p[0] + t_p[1] * t_p[1] + t_p[2] * t_p[2]);
        if (!(n > 0.0) || !isfinite(n)) fail(CSL_ERR_INVALID_ARG, "t_p must be a nonzero vector");
        if (!(alpha >= 0.0 && alpha <= M_PI / 2)) fail(CSL_ERR_INVALID_ARG, "alpha in [0, pi/2]");
        cudaStream_t s = (cudaStream_t)stream;
        SupportConst c;
        c.tx = t_p[0] / n;
        c.ty = t_p[1] / n;
        c.tz = t_p[2] / n;
        c.alpha = alpha;
        static const double paper_a[6] = {-0.02, -0.31, 1.44, -1.11, 0.58, -0.16};
        for (int i = 0; i < 6; ++i) c.a[i] = coeffs ? coeffs[i] : paper_a[i];
        const int n_blocks = 152 * 4;
        DevBuf partial((size_t)n_blocks * 4 * sizeof(double), s), tot(4 * sizeof(double), s);
        k_support<<<n_blocks, kThreads, 0, s>>>(L->nodes.as<float>(), L->edges.as<int32_t>(),
                                                L->radius.as<float>(), L->n_edges, c,
                                                partial.as<double>());
        CSL_LAUNCH_CHECK("support metrics");
        k_support_total<<<1, 32, 0, s>>>(partial.as<double>(), n_blocks, tot.as<double>());
        CSL_LAUNCH_CHECK("support total");
        double h[4];
        read_to_host(h, tot.get(), sizeof(h), s);
        *gamma = h[1] > 0.0 ? h[0] / h[1] : 0.0;
        *psi = h[3] > 0.0 ? 100.0 * h[2] / h[3] : 0.0;
        return CSL_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (...) {
        set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}
