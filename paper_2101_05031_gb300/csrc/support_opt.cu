// Vertex position optimisation for self-support (Sec. 5.3.2, Eq. 16-17).
//
// Every interior vertex of a tetrahedral mesh moves to lower
//   J(v) = sum_{e at v} r_e L_e g(theta_e) / sum_{e at v} r_e L_e     (Eq. 16)
// (theta_e = arccos |u_e . t_P|, Eq. 11; g of Eq. 12, 0 for theta <= alpha)
// inside the inscribed sphere of its star (Eq. 17). The paper visits the
// vertices one by one; here a greedy colouring (vertex order, smallest colour
// free among the neighbours) orders them colour by colour. Vertices of one
// colour share no edge, so each colour is one kernel launch with a warp per
// vertex, and the result equals the sequential sweep in that order.
//
// A move goes along -grad J by step * tau0 (tau0: the smallest distance from
// the vertex's initial position o to the faces opposite it), halved up to
// `backtracks` times until the position lies in the ball |p - o| <= ball *
// tau0, every incident tetrahedron keeps its orientation and min_volume of its
// initial volume, and J decreases. Rounds repeat until nothing moves. All
// arithmetic is FP64 in one fixed order (the build compiles device code with
// --fmad=false).
#include <math.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <vector>

#include "common.cuh"

namespace csl {
namespace {

constexpr int kPoThreads = 128;

struct PoConst {
    double tx, ty, tz, alpha;
    double a[6];
    double step, ball, min_volume;
    int32_t backtracks;
};

// g(theta) of Eq. 12 and its derivative, by Horner (0, 0 for theta <= alpha).
__device__ __forceinline__ void g_dg(double th, const PoConst& c, double& g, double& dg) {
    g = 0.0;
    dg = 0.0;
    if (th <= c.alpha) return;
    for (int i = 5; i >= 0; --i) {
        dg = dg * th + g;
        g = g * th + c.a[i];
    }
}

// One warp evaluates J(v) at (vx, vy, vz) over the vertex's edges [b, e) of
// the CSR: each lane computes the terms of its edges, then the sums are taken
// in edge order (lane by lane through shuffles), the order of the sequential
// definition. With grad != nullptr also the gradient. Every lane returns the
// same values.
__device__ double warp_J(double vx, double vy, double vz, const int32_t* __restrict__ nbr,
                         const double* __restrict__ rad, int64_t b, int64_t e,
                         const double* __restrict__ pos, const PoConst& c, double* grad) {
    const int lane = threadIdx.x & 31;
    double N = 0.0, D = 0.0;
    double dN[3] = {0.0, 0.0, 0.0}, dD[3] = {0.0, 0.0, 0.0};
    const double tk[3] = {c.tx, c.ty, c.tz};
    for (int64_t base = b; base < e; base += 32) {
        const int64_t i = base + lane;
        double tN = 0.0, tD = 0.0, tdN[3] = {0.0, 0.0, 0.0}, tdD[3] = {0.0, 0.0, 0.0};
        bool live = false;
        if (i < e) {
            const int32_t w = nbr[i];
            const double r = rad[i];
            const double d[3] = {vx - pos[3 * (int64_t)w], vy - pos[3 * (int64_t)w + 1],
                                 vz - pos[3 * (int64_t)w + 2]};
            const double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (L != 0.0) {
                live = true;
                const double s = d[0] * c.tx + d[1] * c.ty + d[2] * c.tz;
                const double cs = fmin(fabs(s) / L, 1.0);
                const double th = acos(cs);
                double g, dg;
                g_dg(th, c, g, dg);
                const double dL[3] = {d[0] / L, d[1] / L, d[2] / L};
                tN = r * L * g;
                tD = r * L;
                if (grad) {
                    for (int k = 0; k < 3; ++k) tdD[k] = r * dL[k];
                    if (g != 0.0 || dg != 0.0) {
                        const double sg = copysign(1.0, s);
                        const double s2 = sqrt(fmax(1.0 - cs * cs, 1e-300));
                        for (int k = 0; k < 3; ++k) {
                            const double dc = (sg * tk[k] - cs * dL[k]) / L;
                            const double dth = -dc / s2;
                            tdN[k] = r * (dL[k] * g + L * dg * dth);
                        }
                    }
                }
            }
        }
        const int n = (int)min((int64_t)32, e - base);
        const unsigned live_mask = __ballot_sync(0xffffffffu, live);
        for (int j = 0; j < n; ++j) {   // edge order
            const double xN = __shfl_sync(0xffffffffu, tN, j);
            const double xD = __shfl_sync(0xffffffffu, tD, j);
            double xdN[3], xdD[3];
            if (grad)
                for (int k = 0; k < 3; ++k) {
                    xdN[k] = __shfl_sync(0xffffffffu, tdN[k], j);
                    xdD[k] = __shfl_sync(0xffffffffu, tdD[k], j);
                }
            if (!((live_mask >> j) & 1u)) continue;   // a zero-length edge adds nothing
            N += xN;
            D += xD;
            if (grad)
                for (int k = 0; k < 3; ++k) {
                    dD[k] += xdD[k];
                    dN[k] += xdN[k];
                }
        }
    }
    if (D == 0.0) {
        if (grad) grad[0] = grad[1] = grad[2] = 0.0;
        return 0.0;
    }
    if (grad)
        for (int k = 0; k < 3; ++k) grad[k] = (dN[k] * D - N * dD[k]) / (D * D);
    return N / D;
}

__device__ __forceinline__ double orient(const double* a, const double* b, const double* c,
                                         const double* d) {
    const double ax = b[0] - a[0], ay = b[1] - a[1], az = b[2] - a[2];
    const double bx = c[0] - a[0], by = c[1] - a[1], bz = c[2] - a[2];
    const double cx = d[0] - a[0], cy = d[1] - a[1], cz = d[2] - a[2];
    return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
}

__device__ __forceinline__ double plane_distance(const double* p, const double* a,
                                                 const double* b, const double* c) {
    const double ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
    const double wx = c[0] - a[0], wy = c[1] - a[1], wz = c[2] - a[2];
    const double nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
    const double nn = sqrt(nx * nx + ny * ny + nz * nz);
    if (nn == 0.0) return 0.0;
    const double px = p[0] - a[0], py = p[1] - a[1], pz = p[2] - a[2];
    return fabs(px * nx + py * ny + pz * nz) / nn;
}

__constant__ int kFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

// tau0 of every listed vertex (smallest distance to the faces opposite it)
// and vol0 of every tetrahedron, on the initial mesh.
__global__ void k_po_tau0(const int32_t* __restrict__ list, int64_t n, const double* __restrict__ pos,
                          const int4* __restrict__ tets, const int64_t* __restrict__ vt_off,
                          const int32_t* __restrict__ vt, double* __restrict__ tau0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[i];
        double best = INFINITY;
        for (int64_t q = vt_off[v]; q < vt_off[v + 1]; ++q) {
            const int32_t ti = vt[q] >> 2, k = vt[q] & 3;
            const int4 t = tets[ti];
            const int32_t id[4] = {t.x, t.y, t.z, t.w};
            const double d = plane_distance(pos + 3 * (int64_t)v, pos + 3 * (int64_t)id[kFace[k][0]],
                                            pos + 3 * (int64_t)id[kFace[k][1]],
                                            pos + 3 * (int64_t)id[kFace[k][2]]);
            best = fmin(best, d);
        }
        tau0[v] = best;
    }
}

__global__ void k_po_vol0(const int4* __restrict__ tets, int64_t n, const double* __restrict__ pos,
                          double* __restrict__ vol0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int4 t = tets[i];
        vol0[i] = orient(pos + 3 * (int64_t)t.x, pos + 3 * (int64_t)t.y, pos + 3 * (int64_t)t.z,
                         pos + 3 * (int64_t)t.w);
    }
}

// One colour: a warp per vertex of the list (no two share an edge). The
// lanes share the edge terms and the incident tetrahedra's checks; the trials
// of the backtracking run in order.
//
// A vertex's move depends only on its own position and its neighbours' (all
// the vertices of its tetrahedra) besides constants; so a vertex that did not
// move at its last visit (calm_at: that colour step) and whose star has not
// moved since (moved_at of it and of its neighbours older than that step)
// would not move now either, and is skipped: the result of the sequential
// sweep exactly, without re-evaluating the calm part of the mesh.
__global__ void __launch_bounds__(kPoThreads)
k_po_move(const int32_t* __restrict__ list, int64_t n, double* __restrict__ pos,
          const double* __restrict__ o, const double* __restrict__ tau0,
          const int64_t* __restrict__ e_off, const int32_t* __restrict__ nbr,
          const double* __restrict__ rad, const int64_t* __restrict__ vt_off,
          const int32_t* __restrict__ vt, const int4* __restrict__ tets,
          const double* __restrict__ vol0, PoConst c, int32_t step,
          int32_t* __restrict__ moved_at, int32_t* __restrict__ calm_at, unsigned int* moves) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int32_t v = list[i];
        const int64_t eb = e_off[v], ee = e_off[v + 1];
        const int32_t ca = calm_at[v];
        if (ca >= 0 && moved_at[v] < ca) {   // calm before: has the star moved since?
            bool moved = false;
            for (int64_t q = eb + lane; q < ee; q += 32) moved |= moved_at[nbr[q]] > ca;
            if (!__any_sync(0xffffffffu, moved)) continue;
        }
        double* pv = pos + 3 * (int64_t)v;
        const double p0 = pv[0], p1 = pv[1], p2 = pv[2];
        double grad[3];
        const double J0 = warp_J(p0, p1, p2, nbr, rad, eb, ee, pos, c, grad);
        const double gn = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
        bool went = false;
        if (gn == 0.0) {
            if (lane == 0) calm_at[v] = step;
            continue;
        }
        const double u[3] = {grad[0] / gn, grad[1] / gn, grad[2] / gn};
        const double* ov = o + 3 * (int64_t)v;
        const double rb = c.ball * tau0[v];
        const int64_t tb = vt_off[v], te = vt_off[v + 1];
        double s = c.step * tau0[v];
        for (int it = 0; it <= c.backtracks; ++it, s *= 0.5) {
            const double cand[3] = {p0 - s * u[0], p1 - s * u[1], p2 - s * u[2]};
            const double dx = cand[0] - ov[0], dy = cand[1] - ov[1], dz = cand[2] - ov[2];
            if (sqrt(dx * dx + dy * dy + dz * dz) > rb) continue;
            bool ok = true;
            for (int64_t q = tb + lane; q < te; q += 32) {
                const int32_t ti = vt[q] >> 2, k = vt[q] & 3;
                const int4 t = tets[ti];
                const int32_t id[4] = {t.x, t.y, t.z, t.w};
                const double* P[4];
                for (int j = 0; j < 4; ++j) P[j] = j == k ? cand : pos + 3 * (int64_t)id[j];
                const double vol = orient(P[0], P[1], P[2], P[3]);
                ok = ok && vol * vol0[ti] > 0.0 && fabs(vol) >= c.min_volume * fabs(vol0[ti]);
            }
            if (!__all_sync(0xffffffffu, ok)) continue;
            const double J1 = warp_J(cand[0], cand[1], cand[2], nbr, rad, eb, ee, pos, c, nullptr);
            if (J1 < J0) {
                __syncwarp();   // every lane has read pv before lane 0 writes it
                if (lane == 0) {
                    pv[0] = cand[0];
                    pv[1] = cand[1];
                    pv[2] = cand[2];
                    moved_at[v] = step;
                    atomicAdd(moves, 1u);
                }
                went = true;
                break;
            }
        }
        if (!went && lane == 0) calm_at[v] = step;
    }
}

// Gamma / Psi sums of Eq. 13-14 over the mesh's edges: per block in a fixed
// tree order, then the blocks in order (deterministic).
__global__ void k_po_metrics(const int2* __restrict__ edges, const double* __restrict__ er,
                             int64_t n, const double* __restrict__ pos, PoConst c,
                             double* __restrict__ partial) {
    __shared__ double s[4][kPoThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // r L g (unsupported), r L, L (supported), L
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[i];
        const double* a = pos + 3 * (int64_t)e.x;
        const double* b = pos + 3 * (int64_t)e.y;
        const double d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
        const double L = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double cs = L > 0.0 ? fmin(fabs(d0 * c.tx + d1 * c.ty + d2 * c.tz) / L, 1.0) : 0.0;
        const double th = acos(cs);
        double g, dg;
        g_dg(th, c, g, dg);
        if (th <= c.alpha)
            acc[2] += L;
        else
            acc[0] += er[i] * L * g;
        acc[1] += er[i] * L;
        acc[3] += L;
    }
    for (int k = 0; k < 4; ++k) s[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kPoThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partial[4 * blockIdx.x + k] = s[k][0];
}

__global__ void k_po_metrics_total(const double* __restrict__ partial, int nb, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 4; ++k) t[k] += partial[4 * b + k];
    for (int k = 0; k < 4; ++k) out[k] = t[k];
}

void metrics(const DevBuf& edges, const DevBuf& er, int64_t n_e, const DevBuf& pos,
             const PoConst& c, DevBuf& partial, DevBuf& tot, cudaStream_t s, double* gamma,
             double* psi) {
    const int nb = 152 * 2;
    k_po_metrics<<<nb, kPoThreads, 0, s>>>(edges.as<int2>(), er.as<double>(), n_e, pos.as<double>(),
                                           c, partial.as<double>());
    CSL_LAUNCH_CHECK("support metrics partials");
    k_po_metrics_total<<<1, 32, 0, s>>>(partial.as<double>(), nb, tot.as<double>());
    CSL_LAUNCH_CHECK("support metrics total");
    double h[4];
    read_to_host(h, tot.get(), sizeof(h), s);
    *gamma = h[1] > 0.0 ? h[0] / h[1] : 0.0;
    *psi = h[3] > 0.0 ? 100.0 * h[2] / h[3] : 0.0;
}

template <class T>
void upload(DevBuf& d, const std::vector<T>& h, cudaStream_t s) {
    d.ensure(std::max<size_t>(h.size() * sizeof(T), 16), s);
    if (!h.empty())
        CSL_CUDA(cudaMemcpyAsync(d.get(), h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_support_optimize(float* nodes, int64_t n_nodes, const int32_t* tets,
                                           int64_t n_tets, const float* radius,
                                           const csl_po_params* p, void* stream,
                                           csl_po_result* out, int32_t* moves_per_round) {
    try {
        using clk = std::chrono::steady_clock;
        const auto t_start = clk::now();
        if (!p || !out) fail(CSL_ERR_INVALID_ARG, "NULL argument");
        if (n_nodes < 0 || n_tets < 0) fail(CSL_ERR_INVALID_ARG, "negative count");
        if ((n_nodes && !nodes) || (n_tets && !tets)) fail(CSL_ERR_INVALID_ARG, "NULL array");
        if (n_nodes >= (1ll << 30) || n_tets >= (1ll << 29))
            fail(CSL_ERR_CAPACITY, "too many nodes or tetrahedra");
        const double tn = sqrt(p->t_p[0] * p->t_p[0] + p->t_p[1] * p->t_p[1] + p->t_p[2] * p->t_p[2]);
        if (!(tn > 0.0) || !isfinite(tn)) fail(CSL_ERR_INVALID_ARG, "t_p must be a nonzero vector");
        if (!(p->alpha >= 0.0 && p->alpha <= M_PI / 2)) fail(CSL_ERR_INVALID_ARG, "alpha in [0, pi/2]");
        if (!(p->step > 0.0) || !(p->ball > 0.0) || !isfinite(p->step) || !isfinite(p->ball))
            fail(CSL_ERR_INVALID_ARG, "step and ball must be > 0");
        if (!(p->min_volume >= 0.0 && p->min_volume < 1.0))
            fail(CSL_ERR_INVALID_ARG, "min_volume in [0, 1)");
        if (p->backtracks < 0 || p->backtracks > 60) fail(CSL_ERR_INVALID_ARG, "backtracks in [0, 60]");
        if (p->max_rounds < 0 || p->max_rounds > 100000) fail(CSL_ERR_INVALID_ARG, "max_rounds in [0, 1e5]");
        for (int i = 0; i < 6; ++i)
            if (!isfinite(p->a[i])) fail(CSL_ERR_INVALID_ARG, "non-finite coefficient");
        for (int64_t i = 0; i < 3 * n_nodes; ++i)
            if (!isfinite(nodes[i])) fail(CSL_ERR_INVALID_ARG, "non-finite node coordinate");
        for (int64_t i = 0; i < 4 * n_tets; ++i)
            if (tets[i] < 0 || tets[i] >= n_nodes) fail(CSL_ERR_INVALID_ARG, "node index out of range");

        PoConst c;
        c.tx = p->t_p[0] / tn;
        c.ty = p->t_p[1] / tn;
        c.tz = p->t_p[2] / tn;
        c.alpha = p->alpha;
        for (int i = 0; i < 6; ++i) c.a[i] = p->a[i];
        c.step = p->step;
        c.ball = p->ball;
        c.min_volume = p->min_volume;
        c.backtracks = p->backtracks;
        cudaStream_t s = (cudaStream_t)stream;

        // vertex -> (tetrahedron, corner)
        std::vector<int64_t> vt_off(n_nodes + 1, 0);
        for (int64_t i = 0; i < 4 * n_tets; ++i) ++vt_off[tets[i] + 1];
        for (int64_t v = 0; v < n_nodes; ++v) vt_off[v + 1] += vt_off[v];
        std::vector<int32_t> vt(vt_off[n_nodes]);
        {
            std::vector<int64_t> fill(vt_off.begin(), vt_off.end() - 1);
            for (int64_t t = 0; t < n_tets; ++t)
                for (int k = 0; k < 4; ++k) vt[fill[tets[4 * t + k]]++] = (int32_t)(t * 4 + k);
        }
        // per vertex, its distinct neighbours in ascending order (the edges are
        // then the pairs (v, w > v) in (v, w) order), and its boundary faces:
        // a face (v < b < c) is on the boundary when one tetrahedron has it
        std::vector<int64_t> e_off(n_nodes + 1, 0);
        std::vector<int32_t> nbr;
        nbr.reserve((size_t)n_tets * 4);
        std::vector<uint8_t> fixed(n_nodes, 0);
        std::vector<int64_t> up_off(n_nodes + 1, 0);   // edges (v, w > v) start at up_off[v]
        {
            std::vector<int32_t> tmp;
            std::vector<uint64_t> faces;
            std::vector<int64_t> stamp(n_nodes, -1);   // stamp[w] == v: w already listed for v
            for (int64_t v = 0; v < n_nodes; ++v) {
                tmp.clear();
                faces.clear();
                for (int64_t q = vt_off[v]; q < vt_off[v + 1]; ++q) {
                    const int32_t* tv = tets + 4 * (int64_t)(vt[q] >> 2);
                    const int k = vt[q] & 3;
                    for (int j = 0; j < 4; ++j)
                        if (j != k && tv[j] != v && stamp[tv[j]] != v) {
                            stamp[tv[j]] = v;
                            tmp.push_back(tv[j]);
                        }
                    for (int f = 0; f < 4; ++f) {   // faces containing v as their smallest id
                        if (f == k) continue;
                        int32_t o[2];
                        int m = 0;
                        bool smallest = true;
                        for (int j = 0; j < 4; ++j) {
                            if (j == f || j == k) continue;
                            o[m++] = tv[j];
                            smallest = smallest && tv[j] > v;
                        }
                        if (smallest)
                            faces.push_back(((uint64_t)(uint32_t)std::min(o[0], o[1]) << 32) |
                                            (uint32_t)std::max(o[0], o[1]));
                    }
                }
                std::sort(tmp.begin(), tmp.end());
                nbr.insert(nbr.end(), tmp.begin(), tmp.end());
                e_off[v + 1] = (int64_t)nbr.size();
                up_off[v + 1] = up_off[v] + (int64_t)(tmp.end() - std::upper_bound(tmp.begin(), tmp.end(), (int32_t)v));
                std::sort(faces.begin(), faces.end());
                for (size_t i = 0; i < faces.size();) {
                    size_t j = i;
                    while (j < faces.size() && faces[j] == faces[i]) ++j;
                    if (j - i == 1) {
                        fixed[v] = 1;
                        fixed[(int32_t)(faces[i] >> 32)] = 1;
                        fixed[(int32_t)(faces[i] & 0xffffffffu)] = 1;
                    }
                    i = j;
                }
            }
        }
        const int64_t n_e = up_off[n_nodes];
        std::vector<int2> h_edges(n_e);
        std::vector<double> h_er(n_e);
        for (int64_t v = 0; v < n_nodes; ++v) {
            int64_t id = up_off[v];
            for (int64_t q = e_off[v]; q < e_off[v + 1]; ++q)
                if (nbr[q] > v) {
                    h_edges[id] = make_int2((int32_t)v, nbr[q]);
                    h_er[id] = radius ? (double)radius[id] : 1.0;
                    if (!(h_er[id] > 0.0) || !isfinite(h_er[id]))
                        fail(CSL_ERR_INVALID_ARG, "radius must be > 0");
                    ++id;
                }
        }
        // the radius of every (vertex, neighbour) entry: its edge is (min, max)
        std::vector<double> rad(nbr.size());
        for (int64_t v = 0; v < n_nodes; ++v)
            for (int64_t q = e_off[v]; q < e_off[v + 1]; ++q) {
                const int32_t w = nbr[q];
                const int32_t a = std::min((int32_t)v, w), b = std::max((int32_t)v, w);
                const int32_t* lo = nbr.data() + e_off[a];
                const int32_t* hi = nbr.data() + e_off[a + 1];
                const int32_t* first_up = std::upper_bound(lo, hi, a);
                const int64_t rank = std::lower_bound(first_up, hi, b) - first_up;
                rad[q] = h_er[up_off[a] + rank];
            }
        // greedy colouring in vertex order
        std::vector<int32_t> col(n_nodes, -1);
        int32_t n_col = 0;
        {
            std::vector<int64_t> seen;   // seen[c] == v: colour c taken by a neighbour of v
            for (int64_t v = 0; v < n_nodes; ++v) {
                for (int64_t q = e_off[v]; q < e_off[v + 1]; ++q) {
                    const int32_t cw = col[nbr[q]];
                    if (cw >= 0) {
                        if ((size_t)cw >= seen.size()) seen.resize(cw + 1, -1);
                        seen[cw] = v;
                    }
                }
                int32_t cc = 0;
                while ((size_t)cc < seen.size() && seen[cc] == v) ++cc;
                col[v] = cc;
                n_col = std::max(n_col, cc + 1);
            }
        }
        std::vector<int64_t> col_off(n_col + 1, 0);
        for (int64_t v = 0; v < n_nodes; ++v)
            if (!fixed[v]) ++col_off[col[v] + 1];
        for (int32_t k = 0; k < n_col; ++k) col_off[k + 1] += col_off[k];
        std::vector<int32_t> list(col_off[n_col]);
        {
            std::vector<int64_t> fill(col_off.begin(), col_off.end() - 1);
            for (int64_t v = 0; v < n_nodes; ++v)
                if (!fixed[v]) list[fill[col[v]]++] = (int32_t)v;
        }

        const double host_ms =
            std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
        std::vector<double> h_pos(3 * n_nodes);
        for (int64_t i = 0; i < 3 * n_nodes; ++i) h_pos[i] = (double)nodes[i];
        std::vector<int4> h_tets(n_tets);
        for (int64_t t = 0; t < n_tets; ++t)
            h_tets[t] = make_int4(tets[4 * t], tets[4 * t + 1], tets[4 * t + 2], tets[4 * t + 3]);
        DevBuf d_pos, d_o, d_tau, d_eoff, d_nbr, d_rad, d_vtoff, d_vt, d_tets, d_vol0, d_list;
        DevBuf d_edges, d_er, d_part((size_t)152 * 2 * 4 * sizeof(double), s), d_tot(64, s);
        DevBuf d_moves(16, s);
        // colour step of each vertex's last move and of its last visit without one
        DevBuf d_moved_at(std::max<size_t>((size_t)n_nodes * 4, 16), s),
            d_calm_at(std::max<size_t>((size_t)n_nodes * 4, 16), s);
        CSL_CUDA(cudaMemsetAsync(d_moved_at.get(), 0xff, d_moved_at.size(), s));
        CSL_CUDA(cudaMemsetAsync(d_calm_at.get(), 0xff, d_calm_at.size(), s));
        upload(d_pos, h_pos, s);
        upload(d_o, h_pos, s);
        upload(d_eoff, e_off, s);
        upload(d_nbr, nbr, s);
        upload(d_rad, rad, s);
        upload(d_vtoff, vt_off, s);
        upload(d_vt, vt, s);
        upload(d_tets, h_tets, s);
        upload(d_list, list, s);
        upload(d_edges, h_edges, s);
        upload(d_er, h_er, s);
        d_tau.ensure(std::max<size_t>((size_t)n_nodes * 8, 16), s);
        d_vol0.ensure(std::max<size_t>((size_t)n_tets * 8, 16), s);
        const int64_t n_list = (int64_t)list.size();
        if (n_list) {
            k_po_tau0<<<grid_for(n_list, kPoThreads), kPoThreads, 0, s>>>(
                d_list.as<int32_t>(), n_list, d_pos.as<double>(), d_tets.as<int4>(),
                d_vtoff.as<int64_t>(), d_vt.as<int32_t>(), d_tau.as<double>());
            CSL_LAUNCH_CHECK("inscribed radii");
        }
        if (n_tets) {
            k_po_vol0<<<grid_for(n_tets, kPoThreads), kPoThreads, 0, s>>>(
                d_tets.as<int4>(), n_tets, d_pos.as<double>(), d_vol0.as<double>());
            CSL_LAUNCH_CHECK("initial volumes");
        }
        csl_po_result r = {};
        r.n_colours = n_col;
        metrics(d_edges, d_er, n_e, d_pos, c, d_part, d_tot, s, &r.gamma_before, &r.psi_before);
        for (int32_t round = 0; round < p->max_rounds && n_list; ++round) {
            CSL_CUDA(cudaMemsetAsync(d_moves.get(), 0, 4, s));
            for (int32_t k = 0; k < n_col; ++k) {
                const int64_t b = col_off[k], n = col_off[k + 1] - b;
                if (!n) continue;
                k_po_move<<<grid_for(n * 32, kPoThreads), kPoThreads, 0, s>>>(
                    d_list.as<int32_t>() + b, n, d_pos.as<double>(), d_o.as<double>(),
                    d_tau.as<double>(), d_eoff.as<int64_t>(), d_nbr.as<int32_t>(),
                    d_rad.as<double>(), d_vtoff.as<int64_t>(), d_vt.as<int32_t>(),
                    d_tets.as<int4>(), d_vol0.as<double>(), c, round * n_col + k,
                    d_moved_at.as<int32_t>(), d_calm_at.as<int32_t>(), d_moves.as<unsigned int>());
                CSL_LAUNCH_CHECK("vertex moves");
            }
            unsigned int moved = 0;
            read_to_host(&moved, d_moves.get(), 4, s);
            if (moves_per_round) moves_per_round[round] = (int32_t)moved;
            r.moves += moved;
            ++r.rounds;
            if (moved == 0) break;
        }
        metrics(d_edges, d_er, n_e, d_pos, c, d_part, d_tot, s, &r.gamma_after, &r.psi_after);
        if (n_nodes) read_to_host(h_pos.data(), d_pos.get(), h_pos.size() * 8, s);
        for (int64_t i = 0; i < 3 * n_nodes; ++i) nodes[i] = (float)h_pos[i];
        r.host_ms = host_ms;
        r.wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
        *out = r;
        return CSL_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return CSL_ERR_OOM;
    } catch (...) {
        set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}
