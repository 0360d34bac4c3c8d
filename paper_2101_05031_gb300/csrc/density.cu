// Density matching of a tetrahedral lattice (Sec. 5.5): the subdivision and
// radius-tuning operators applied in the paper's four steps.
//
// Device work: the target of every tetrahedron (containment of voxel centres
// by four FP64 determinants, else trilinear interpolation at the centroid),
// its density at n^3 samples with the doubled radius (rho*) and the bisection
// of its radius ratio, the smallest ratio per edge, the voxel-edge pairs (count,
// scan, emit, radix sort by voxel), the per-voxel bisection of a common ratio
// and the per-edge minimum. The topology of the subdivision (new midpoints,
// halves, children, edge numbering) is kept on the device too
// (density_mesh.cu); the host validates the input and copies the result out.
//
// A density depends on the radius only through the weight, so each block
// first sums the unit-weight segment integrals J(p) of the struts being tuned
// (and the fixed part F(p) of the others) at its samples, in shared memory;
// a bisection step is then one weighted sigmoid mean over the samples, reduced
// in a fixed order (deterministic).
#include <math.h>

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "common.cuh"
#include "density_mesh.cuh"
#include "field_tile.cuh"

namespace csl {
namespace {

constexpr int kDmThreads = 256;
constexpr int kDmMaxSamples = 16 * 16 * 16;

struct DmConst {
    double r0, R, C;   // base radius, support, iso-value
    float R2, Cf, inv_T;
    int32_t iters;
};

struct GridConst {
    double ox, oy, oz, h;
    int32_t nx, ny, nz;
};

// PHYSICAL weight over R^4 (Sec. 3.2): Sigma = w_R4(r) * R^4 I.
__device__ __forceinline__ float weight_R4(double r, const DmConst& c) {
    const double q = c.R * c.R - r * r;
    return (float)(15.0 * c.C / (16.0 * q * q * sqrt(q)));
}

// R^4 I of one strut (tile-local frame: start a, unit direction u, length len)
// at p: the segment integral of Eq. 7 with its arc-length factor.
__device__ __forceinline__ float strut_R4I(float px, float py, float pz, float4 a, float4 u,
                                           float R2) {
    const float qx = px - a.x, qy = py - a.y, qz = pz - a.z;
    const float t0 = qx * u.x + qy * u.y + qz * u.z;
    const float ex = qx - t0 * u.x, ey = qy - t0 * u.y, ez = qz - t0 * u.z;
    const float h2 = R2 - (ex * ex + ey * ey + ez * ez);
    if (!(h2 > 0.0f) || !(u.w > 0.0f)) return 0.0f;
    return segment_term_R4(t0, h2, u.w);
}

// Mean of sigma((F + W J - C) / T) over the n samples held in shared memory.
// The same mean by one warp (lane-strided samples, butterfly sum: every lane
// gets the same value, in a fixed order).
__device__ __forceinline__ float warp_mean_density(const float* F, const float* J, int n, float W,
                                                   const DmConst& c) {
    float acc = 0.0f;
    for (int k = threadIdx.x & 31; k < n; k += 32) {
        const float f = F ? F[k] : 0.0f;
        const float x = (f + W * J[k] - c.Cf) * c.inv_T;
        acc += 1.0f / (1.0f + expf(-x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc / (float)n;
}

// The ratio s in [1/2, 2] at which the density reaches `target` (the end
// points when it is out of reach, else `iters` halvings), by one warp;
// *rho_hi = density at s = 2.
__device__ float warp_bisect_ratio(const float* F, const float* J, int n, float target,
                                   const DmConst& c, float* rho_hi) {
    const float r_hi = warp_mean_density(F, J, n, weight_R4(c.r0 * 2.0, c), c);
    *rho_hi = r_hi;
    if (r_hi <= target) return 2.0f;
    if (warp_mean_density(F, J, n, weight_R4(c.r0 * 0.5, c), c) >= target) return 0.5f;
    float lo = 0.5f, hi = 2.0f;
    for (int it = 0; it < c.iters; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (warp_mean_density(F, J, n, weight_R4(c.r0 * (double)mid, c), c) < target)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5f * (lo + hi);
}

// ---- Step 1: targets ----------------------------------------------------

__device__ __forceinline__ double orient(double3 a, double3 b, double3 c, double3 d) {
    const double ax = b.x - a.x, ay = b.y - a.y, az = b.z - a.z;
    const double bx = c.x - a.x, by = c.y - a.y, bz = c.z - a.z;
    const double cx = d.x - a.x, cy = d.y - a.y, cz = d.z - a.z;
    return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
}

__device__ __forceinline__ bool contains(const double3 (&v)[4], double D, double3 p) {
    const double d0 = orient(p, v[1], v[2], v[3]);
    const double d1 = orient(v[0], p, v[2], v[3]);
    const double d2 = orient(v[0], v[1], p, v[3]);
    const double d3 = orient(v[0], v[1], v[2], p);
    if (D > 0.0) return d0 >= 0.0 && d1 >= 0.0 && d2 >= 0.0 && d3 >= 0.0;
    return d0 <= 0.0 && d1 <= 0.0 && d2 <= 0.0 && d3 <= 0.0;
}

__device__ double trilinear(const GridConst& g, const float* __restrict__ tgt, double3 p) {
    const double pc[3] = {p.x, p.y, p.z};
    const double oc[3] = {g.ox, g.oy, g.oz};
    const int dims[3] = {g.nx, g.ny, g.nz};
    int idx[3];
    double f[3];
    for (int ax = 0; ax < 3; ++ax) {
        const int n = dims[ax];
        if (n == 1) {
            idx[ax] = 0;
            f[ax] = 0.0;
            continue;
        }
        double q = (pc[ax] - oc[ax]) / g.h - 0.5;
        q = fmin(fmax(q, 0.0), (double)(n - 1));
        const int i0 = min((int)floor(q), n - 2);
        idx[ax] = i0;
        f[ax] = q - (double)i0;
    }
    double val = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                const double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) *
                                 (cz ? f[2] : 1.0 - f[2]);
                if (w == 0.0) continue;
                const int i = min(idx[0] + cx, g.nx - 1), j = min(idx[1] + cy, g.ny - 1);
                const int k = min(idx[2] + cz, g.nz - 1);
                val += w * (double)tgt[((int64_t)k * g.ny + j) * g.nx + i];
            }
    return val;
}

// Voxel index range [lo, hi] along one axis whose centres may lie in [a, b]
// (one extra voxel on each side; the containment test decides).
__device__ __forceinline__ void centre_range(double a, double b, double o, double h, int n,
                                             int& lo, int& hi) {
    const double fa = fmin(fmax((a - o) / h - 0.5, -2.0), (double)n + 1.0);
    const double fb = fmin(fmax((b - o) / h - 0.5, -2.0), (double)n + 1.0);
    lo = max(0, (int)floor(fa) - 1);
    hi = min(n - 1, (int)ceil(fb) + 1);
}

// One warp per tetrahedron: the largest target of the contained voxel
// centres, else the interpolated target at the centroid.
__global__ void k_dm_target(const float4* __restrict__ tv, int64_t n_tets, GridConst g,
                            const float* __restrict__ tgt, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tets;
         t += warps) {
        double3 v[4];
        for (int k = 0; k < 4; ++k) {
            const float4 q = tv[4 * t + k];
            v[k] = make_double3(q.x, q.y, q.z);
        }
        const double D = orient(v[0], v[1], v[2], v[3]);
        const double xmin = fmin(fmin(v[0].x, v[1].x), fmin(v[2].x, v[3].x));
        const double xmax = fmax(fmax(v[0].x, v[1].x), fmax(v[2].x, v[3].x));
        const double ymin = fmin(fmin(v[0].y, v[1].y), fmin(v[2].y, v[3].y));
        const double ymax = fmax(fmax(v[0].y, v[1].y), fmax(v[2].y, v[3].y));
        const double zmin = fmin(fmin(v[0].z, v[1].z), fmin(v[2].z, v[3].z));
        const double zmax = fmax(fmax(v[0].z, v[1].z), fmax(v[2].z, v[3].z));
        int i0, i1, j0, j1, k0, k1;
        centre_range(xmin, xmax, g.ox, g.h, g.nx, i0, i1);
        centre_range(ymin, ymax, g.oy, g.h, g.ny, j0, j1);
        centre_range(zmin, zmax, g.oz, g.h, g.nz, k0, k1);
        const int64_t ni = i1 - i0 + 1, nj = j1 - j0 + 1, nk = k1 - k0 + 1;
        const int64_t cnt = (D != 0.0 && ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
        double best = -INFINITY;
        bool found = false;
        for (int64_t q = lane; q < cnt; q += 32) {
            const int i = i0 + (int)(q % ni);
            const int j = j0 + (int)((q / ni) % nj);
            const int k = k0 + (int)(q / (ni * nj));
            const double3 p = make_double3(g.ox + g.h * ((double)i + 0.5),
                                           g.oy + g.h * ((double)j + 0.5),
                                           g.oz + g.h * ((double)k + 0.5));
            // a centre outside the bounding box cannot be contained
            const bool in_box = p.x >= xmin && p.x <= xmax && p.y >= ymin && p.y <= ymax &&
                                p.z >= zmin && p.z <= zmax;
            if (in_box && contains(v, D, p)) {
                found = true;
                best = fmax(best, (double)tgt[((int64_t)k * g.ny + j) * g.nx + i]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        found = __any_sync(0xffffffffu, found);
        if (lane == 0) {
            if (found) {
                out[t] = best;
            } else {
                const double3 c = make_double3((v[0].x + v[1].x + v[2].x + v[3].x) * 0.25,
                                               (v[0].y + v[1].y + v[2].y + v[3].y) * 0.25,
                                               (v[0].z + v[1].z + v[2].z + v[3].z) * 0.25);
                out[t] = trilinear(g, tgt, c);
            }
        }
    }
}

// ---- Steps 2 and 3: density of a tetrahedron, rho* and the bisection -----

// One warp per tetrahedron, J(p) of its six struts in the warp's slice of
// dynamic shared memory (n_samples floats). coef: the n^3 Kuhn-centroid
// coefficients; the sample is a1 (v1 - v0) + a2 (v2 - v1) + a3 (v3 - v2)
// relative to v0.
__global__ void __launch_bounds__(kDmThreads)
k_dm_tet(const float4* __restrict__ tv, const double* __restrict__ target, int64_t n_tets,
         const float4* __restrict__ coef, int n_samples, DmConst c, float* __restrict__ rho_star,
         float* __restrict__ ratio) {
    extern __shared__ float s_dyn[];
    const int lane = threadIdx.x & 31;
    float* s_J = s_dyn + (size_t)(threadIdx.x >> 5) * n_samples;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tets;
         t += warps) {
        const float4 v0 = tv[4 * t];
        float3 w[4];
        w[0] = make_float3(0.0f, 0.0f, 0.0f);
        for (int k = 1; k < 4; ++k) {
            const float4 q = tv[4 * t + k];
            w[k] = make_float3(q.x - v0.x, q.y - v0.y, q.z - v0.z);
        }
        float4 ea[6], eu[6];
        const int ep[6] = {0, 0, 0, 1, 1, 2}, eq[6] = {1, 2, 3, 2, 3, 3};   // local edges
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const float3 a = w[ep[e]], b = w[eq[e]];
            const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
            const float len = sqrtf(dx * dx + dy * dy + dz * dz);
            const float il = len > 0.0f ? 1.0f / len : 0.0f;
            ea[e] = make_float4(a.x, a.y, a.z, 0.0f);
            eu[e] = make_float4(dx * il, dy * il, dz * il, len);
        }
        const float3 d1 = w[1];
        const float3 d2 = make_float3(w[2].x - w[1].x, w[2].y - w[1].y, w[2].z - w[1].z);
        const float3 d3 = make_float3(w[3].x - w[2].x, w[3].y - w[2].y, w[3].z - w[2].z);
        for (int k = lane; k < n_samples; k += 32) {
            const float4 a = coef[k];
            const float px = a.x * d1.x + a.y * d2.x + a.z * d3.x;
            const float py = a.x * d1.y + a.y * d2.y + a.z * d3.y;
            const float pz = a.x * d1.z + a.y * d2.z + a.z * d3.z;
            float J = 0.0f;
#pragma unroll
            for (int e = 0; e < 6; ++e) J += strut_R4I(px, py, pz, ea[e], eu[e], c.R2);
            s_J[k] = J;
        }
        __syncwarp();
        float r_hi;
        const float s = warp_bisect_ratio(nullptr, s_J, n_samples, (float)target[t], c, &r_hi);
        if (lane == 0) {
            rho_star[t] = r_hi;
            ratio[t] = s;
        }
        __syncwarp();   // s_J is rewritten by the next tetrahedron
    }
}

// Step 2's decision: a tetrahedron whose rho* stays below its target splits.
__global__ void k_dm_split(const float* __restrict__ rho, const double* __restrict__ target,
                           int64_t n, uint32_t* __restrict__ split) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        split[i] = (double)rho[i] < target[i] ? 1u : 0u;
}

__global__ void k_dm_fill_u32(uint32_t* __restrict__ a, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// An edge in no leaf tetrahedron (none in a consistent mesh) keeps ratio 1.
__global__ void k_dm_ratio_fix(uint32_t* ratio_bits, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (ratio_bits[i] == 0x7f800000u) ratio_bits[i] = __float_as_uint(1.0f);
}

// ---- Step 4: voxels -------------------------------------------------------

// Voxel range of a strut's support box (the segment's box grown by `reach`).
__device__ __forceinline__ bool support_range(float4 a, float4 b, const GridConst& g, double reach,
                                              int& i0, int& i1, int& j0, int& j1, int& k0,
                                              int& k1) {
    const double pa[3] = {a.x, a.y, a.z}, pb[3] = {b.x, b.y, b.z};
    const double o[3] = {g.ox, g.oy, g.oz};
    const int n[3] = {g.nx, g.ny, g.nz};
    int lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) {
        const double l = (fmin(pa[ax], pb[ax]) - reach - o[ax]) / g.h;
        const double h = (fmax(pa[ax], pb[ax]) + reach - o[ax]) / g.h;
        if (h < 0.0 || l >= (double)n[ax]) return false;
        lo[ax] = max(0, (int)floor(fmax(l, -1.0)));
        hi[ax] = min(n[ax] - 1, (int)floor(fmin(h, (double)n[ax])));
    }
    i0 = lo[0]; i1 = hi[0]; j0 = lo[1]; j1 = hi[1]; k0 = lo[2]; k1 = hi[2];
    return true;
}

__global__ void k_dm_vox_count(const float4* __restrict__ sa, const float4* __restrict__ sb,
                               int64_t n_seg, GridConst g, double reach,
                               uint32_t* __restrict__ cnt) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seg;
         s += (int64_t)gridDim.x * blockDim.x) {
        int i0, i1, j0, j1, k0, k1;
        uint64_t c = 0;
        if (support_range(sa[s], sb[s], g, reach, i0, i1, j0, j1, k0, k1))
            c = (uint64_t)(i1 - i0 + 1) * (uint64_t)(j1 - j0 + 1) * (uint64_t)(k1 - k0 + 1);
        cnt[s] = (uint32_t)min(c, (uint64_t)0xffffffffu);
    }
}

// Closed segment a-b against the closed box [lo, hi], slab by slab in FP64.
__device__ __forceinline__ bool seg_meets_box(const double (&a)[3], const double (&b)[3],
                                              const double (&lo)[3], const double (&hi)[3]) {
    double t0 = 0.0, t1 = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double d = b[k] - a[k];
        if (d == 0.0) {
            if (a[k] < lo[k] || a[k] > hi[k]) return false;
        } else {
            double ta = (lo[k] - a[k]) / d;
            double tb = (hi[k] - a[k]) / d;
            if (ta > tb) {
                const double x = ta;
                ta = tb;
                tb = x;
            }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
            if (t0 > t1) return false;
        }
    }
    return true;
}

// keys: voxel id; vals: strut << 1 | (the strut meets the voxel).
__global__ void k_dm_vox_emit(const float4* __restrict__ sa, const float4* __restrict__ sb,
                              int64_t n_seg, GridConst g, double reach,
                              const int64_t* __restrict__ off, uint32_t* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seg;
         s += (int64_t)gridDim.x * blockDim.x) {
        int i0, i1, j0, j1, k0, k1;
        const float4 fa = sa[s], fb = sb[s];
        if (!support_range(fa, fb, g, reach, i0, i1, j0, j1, k0, k1)) continue;
        const double a[3] = {fa.x, fa.y, fa.z}, b[3] = {fb.x, fb.y, fb.z};
        int64_t o = off[s];
        for (int k = k0; k <= k1; ++k)
            for (int j = j0; j <= j1; ++j)
                for (int i = i0; i <= i1; ++i) {
                    const double lo[3] = {g.ox + g.h * (double)i, g.oy + g.h * (double)j,
                                          g.oz + g.h * (double)k};
                    const double hi[3] = {g.ox + g.h * (double)(i + 1), g.oy + g.h * (double)(j + 1),
                                          g.oz + g.h * (double)(k + 1)};
                    keys[o] = (uint32_t)(((int64_t)k * g.ny + j) * g.nx + i);
                    vals[o] = ((uint32_t)s << 1) | (seg_meets_box(a, b, lo, hi) ? 1u : 0u);
                    ++o;
                }
    }
}

// [beg, end) of every voxel's run in the sorted keys (untouched voxels stay 0, 0).
__global__ void k_dm_vox_bounds(const uint32_t* __restrict__ keys, int64_t n,
                                uint32_t* __restrict__ beg, uint32_t* __restrict__ end) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) beg[k] = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) end[k] = (uint32_t)(i + 1);
    }
}

// One block per voxel: F (struts not meeting the voxel, at their Step-3
// radii) and J (struts meeting it, unit weight) at the m^3 samples, then the
// bisection of the common ratio. NaN when no strut meets the voxel.
__global__ void __launch_bounds__(kDmThreads)
k_dm_voxel(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ vbeg,
           const uint32_t* __restrict__ vend, const float4* __restrict__ sa,
           const float4* __restrict__ sb, const float* __restrict__ ratio3,
           const float* __restrict__ tgt, GridConst g, DmConst c, int m,
           float* __restrict__ vox_ratio) {
    __shared__ float s_F[kDmMaxSamples], s_J[kDmMaxSamples];
    __shared__ float4 s_a[kDmThreads], s_u[kDmThreads];
    const int n = m * m * m;
    const int64_t n_vox = (int64_t)g.nx * g.ny * g.nz;
    const float hf = (float)g.h, inv_m = 1.0f / (float)m;
    for (int64_t v = blockIdx.x; v < n_vox; v += gridDim.x) {
        const uint32_t b0 = vbeg[v], b1 = vend[v];
        if (b0 >= b1) {
            if (threadIdx.x == 0) vox_ratio[v] = __int_as_float(0x7fc00000);
            continue;
        }
        const int i = (int)(v % g.nx), j = (int)((v / g.nx) % g.ny), k = (int)(v / ((int64_t)g.nx * g.ny));
        const double cx = g.ox + g.h * (double)i, cy = g.oy + g.h * (double)j,
                     cz = g.oz + g.h * (double)k;
        for (int q = threadIdx.x; q < n; q += kDmThreads) {
            s_F[q] = 0.0f;
            s_J[q] = 0.0f;
        }
        int any_meet = 0;
        for (uint32_t c0 = b0; c0 < b1; c0 += kDmThreads) {
            const int cnt = (int)min((uint32_t)kDmThreads, b1 - c0);
            if ((int)threadIdx.x < cnt) {
                const uint32_t pv = vals[c0 + threadIdx.x];
                const uint32_t s = pv >> 1;
                const float4 fa = sa[s], fb = sb[s];
                const float ax = (float)((double)fa.x - cx), ay = (float)((double)fa.y - cy),
                            az = (float)((double)fa.z - cz);
                const float dx = (float)((double)fb.x - cx) - ax, dy = (float)((double)fb.y - cy) - ay,
                            dz = (float)((double)fb.z - cz) - az;
                const float len = sqrtf(dx * dx + dy * dy + dz * dz);
                const float il = len > 0.0f ? 1.0f / len : 0.0f;
                // w < 0 marks a strut that meets the voxel (tuned, unit weight)
                const float W = (pv & 1u) ? -1.0f : weight_R4(c.r0 * (double)ratio3[s], c);
                s_a[threadIdx.x] = make_float4(ax, ay, az, W);
                s_u[threadIdx.x] = make_float4(dx * il, dy * il, dz * il, len);
            }
            any_meet |= __syncthreads_or((int)threadIdx.x < cnt && (vals[c0 + threadIdx.x] & 1u));
            for (int q = threadIdx.x; q < n; q += kDmThreads) {
                const int qx = q % m, qy = (q / m) % m, qz = q / (m * m);
                const float px = hf * (((float)qx + 0.5f) * inv_m);
                const float py = hf * (((float)qy + 0.5f) * inv_m);
                const float pz = hf * (((float)qz + 0.5f) * inv_m);
                float F = s_F[q], J = s_J[q];
                for (int r = 0; r < cnt; ++r) {
                    const float4 a = s_a[r];
                    const float term = strut_R4I(px, py, pz, a, s_u[r], c.R2);
                    if (a.w < 0.0f)
                        J += term;
                    else
                        F += a.w * term;
                }
                s_F[q] = F;
                s_J[q] = J;
            }
            __syncthreads();
        }
        if (!any_meet) {
            if (threadIdx.x == 0) vox_ratio[v] = __int_as_float(0x7fc00000);
            continue;
        }
        if (threadIdx.x < 32) {   // one warp bisects; no block barrier per step
            float r_hi;
            const float s = warp_bisect_ratio(s_F, s_J, n, tgt[v], c, &r_hi);
            if (threadIdx.x == 0) vox_ratio[v] = s;
        }
        __syncthreads();   // s_F, s_J are rewritten by the next voxel
    }
}

// Step 4's rule per (voxel, meeting strut) pair: the smaller ratio.
__global__ void k_dm_vox_min(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                             int64_t n, const float* __restrict__ vox_ratio, uint32_t* ratio_bits) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = vals[i];
        if (v & 1u) atomicMin(ratio_bits + (v >> 1), __float_as_uint(vox_ratio[keys[i]]));
    }
}

__global__ void k_dm_radii(const float* __restrict__ ratio, int64_t n, float r0,
                           float* __restrict__ radius) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        radius[i] = r0 * ratio[i];
}

// Centroids of the n-fold Kuhn subdivision of {1 >= x1 >= x2 >= x3 >= 0}:
// the cube cells' simplices c + (3 e_a + 2 e_b + e_c) / 4 that lie in it.
std::vector<float4> kuhn_table(int n) {
    std::vector<float4> out;
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                for (const auto& p : perms) {
                    double x[3] = {(double)i, (double)j, (double)k};
                    x[p[0]] += 0.75;
                    x[p[1]] += 0.5;
                    x[p[2]] += 0.25;
                    if (x[0] > x[1] && x[1] > x[2])
                        out.push_back(make_float4((float)(x[0] / n), (float)(x[1] / n),
                                                  (float)(x[2] / n), 0.0f));
                }
    if ((int64_t)out.size() != (int64_t)n * n * n) fail(CSL_ERR_CUDA, "Kuhn table size");
    return out;
}

// Accumulates the time spent between start() and stop() calls.
struct HostClock {
    using clock = std::chrono::steady_clock;
    double ms = 0.0;
    clock::time_point t0;
    void start() { t0 = clock::now(); }
    void stop() { ms += std::chrono::duration<double, std::milli>(clock::now() - t0).count(); }
};

template <class T>
void upload(DevBuf& d, const std::vector<T>& h, cudaStream_t s) {
    d.ensure(std::max<size_t>(h.size() * sizeof(T), 16), s);
    if (!h.empty())
        CSL_CUDA(cudaMemcpyAsync(d.get(), h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

template <class T>
void download(std::vector<T>& h, const DevBuf& d, size_t n, cudaStream_t s) {
    h.resize(n);
    if (n) read_to_host(h.data(), d.get(), n * sizeof(T), s);
}

void* host_copy(const void* src, size_t bytes) {
    void* p = host_block_alloc(bytes ? bytes : 16);
    if (!p) fail(CSL_ERR_OOM, "host result block");
    if (bytes) memcpy(p, src, bytes);
    return p;
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_density_match(const float* nodes, int64_t n_nodes, const int32_t* tets,
                                        int64_t n_tets, const csl_voxels* vox,
                                        const csl_dm_params* p, void* stream,
                                        csl_dm_result** out) {
    try {
        HostClock wall, host;
        wall.start();
        host.start();
        if (!out || !vox || !p) fail(CSL_ERR_INVALID_ARG, "NULL argument");
        *out = nullptr;
        if (n_nodes < 0 || n_tets < 0) fail(CSL_ERR_INVALID_ARG, "negative count");
        if ((n_nodes && !nodes) || (n_tets && !tets)) fail(CSL_ERR_INVALID_ARG, "NULL array");
        if (n_nodes >= (1ll << 30) || n_tets >= (1ll << 27))
            fail(CSL_ERR_CAPACITY, "too many nodes or tetrahedra");
        if (!(p->r_min > 0.0f) || !isfinite(p->r_min)) fail(CSL_ERR_INVALID_ARG, "r_min must be > 0");
        const double r0 = 2.0 * (double)p->r_min;
        const double R = p->R == 0.0f ? 3.0 * r0 : (double)p->R;
        if (!(R > 2.0 * r0) || !isfinite(R))
            fail(CSL_ERR_INVALID_ARG, "R must exceed the doubled base radius 4 r_min");
        if (!(p->C > 0.0f) || !isfinite(p->C)) fail(CSL_ERR_INVALID_ARG, "C must be > 0");
        if (!(p->temperature > 0.0f) || !isfinite(p->temperature))
            fail(CSL_ERR_INVALID_ARG, "temperature must be > 0");
        if (p->tet_n < 1 || p->tet_n > 16 || p->vox_m < 1 || p->vox_m > 16)
            fail(CSL_ERR_INVALID_ARG, "tet_n and vox_m in [1, 16]");
        if (p->max_depth < 0 || p->max_depth > 8) fail(CSL_ERR_INVALID_ARG, "max_depth in [0, 8]");
        if (p->iters < 1 || p->iters > 40) fail(CSL_ERR_INVALID_ARG, "iters in [1, 40]");
        if (!(vox->h > 0.0) || !isfinite(vox->h)) fail(CSL_ERR_INVALID_ARG, "voxel h must be > 0");
        for (int k = 0; k < 3; ++k) {
            if (!isfinite(vox->origin[k])) fail(CSL_ERR_INVALID_ARG, "non-finite voxel origin");
            if (vox->dims[k] < 1) fail(CSL_ERR_INVALID_ARG, "voxel dims must be >= 1");
        }
        const int64_t n_vox = (int64_t)vox->dims[0] * vox->dims[1] * vox->dims[2];
        if (n_vox >= (1ll << 31)) fail(CSL_ERR_CAPACITY, "too many voxels");
        if (!vox->target) fail(CSL_ERR_INVALID_ARG, "NULL target");
        for (int64_t i = 0; i < n_vox; ++i)
            if (!isfinite(vox->target[i])) fail(CSL_ERR_INVALID_ARG, "non-finite target");
        for (int64_t i = 0; i < 3 * n_nodes; ++i)
            if (!isfinite(nodes[i])) fail(CSL_ERR_INVALID_ARG, "non-finite node coordinate");
        for (int64_t i = 0; i < 4 * n_tets; ++i)
            if (tets[i] < 0 || tets[i] >= n_nodes) fail(CSL_ERR_INVALID_ARG, "node index out of range");

        cudaStream_t s = (cudaStream_t)stream;
        DmConst c;
        c.r0 = r0;
        c.R = R;
        c.C = (double)p->C;
        c.R2 = (float)(R * R);
        c.Cf = p->C;
        c.inv_T = (float)(1.0 / ((double)p->temperature * (double)p->C));
        c.iters = p->iters;
        GridConst g;
        g.ox = vox->origin[0];
        g.oy = vox->origin[1];
        g.oz = vox->origin[2];
        g.h = vox->h;
        g.nx = vox->dims[0];
        g.ny = vox->dims[1];
        g.nz = vox->dims[2];
        const int n_samples = p->tet_n * p->tet_n * p->tet_n;
        // warps per block of the tetrahedron kernel: their J slices fit 48 KB
        const int tet_warps = std::max(1, std::min(kDmThreads / 32, 12288 / n_samples));
        const int tet_threads = 32 * tet_warps;
        const size_t tet_smem = (size_t)tet_warps * n_samples * sizeof(float);

        // the mesh on the device: its edges numbered in (smaller, larger) node order
        host.stop();
        DevMesh mesh;
        mesh_init(mesh, nodes, n_nodes, tets, n_tets, s);
        DevBuf d_tgt((size_t)n_vox * sizeof(float), s);
        CSL_CUDA(cudaMemcpyAsync(d_tgt.get(), vox->target, (size_t)n_vox * sizeof(float),
                                 cudaMemcpyHostToDevice, s));
        DevBuf d_coef;
        upload(d_coef, kuhn_table(p->tet_n), s);

        // Steps 1-3 level by level on the device: targets, rho* and the ratio of
        // the level's tetrahedra (the input, then the children of the last
        // level's splits: a contiguous range of ids), then the subdivision.
        // Values are kept per tetrahedron id.
        DevBuf d_target, d_rho, d_ratio, d_tv, d_split;
        auto per_tet = [&](int64_t used, int64_t need) {
            auto keep = [&](DevBuf& b, size_t el) {
                if ((size_t)need * el <= b.size()) return;
                DevBuf nb((size_t)std::max<int64_t>(need, 1) * el, s);
                if (used)
                    CSL_CUDA(cudaMemcpyAsync(nb.get(), b.get(), (size_t)used * el,
                                             cudaMemcpyDeviceToDevice, s));
                b = std::move(nb);
            };
            keep(d_target, sizeof(double));
            keep(d_rho, sizeof(float));
            keep(d_ratio, sizeof(float));
        };
        per_tet(0, n_tets);
        int64_t n_split = 0, t0 = 0, nc = n_tets;
        for (int d = 0; d <= p->max_depth && nc > 0; ++d) {
            d_tv.ensure((size_t)nc * 4 * sizeof(float4), s);
            mesh_corners(mesh, t0, nc, d_tv.as<float4>(), s);
            double* tgt_d = d_target.as<double>() + t0;
            float* rho_d = d_rho.as<float>() + t0;
            float* rat_d = d_ratio.as<float>() + t0;
            k_dm_target<<<grid_for(nc * 32, 256), 256, 0, s>>>(d_tv.as<float4>(), nc, g,
                                                               d_tgt.as<float>(), tgt_d);
            CSL_LAUNCH_CHECK("density targets");
            k_dm_tet<<<grid_for(nc * 32, tet_threads), tet_threads, tet_smem, s>>>(
                d_tv.as<float4>(), tgt_d, nc, d_coef.as<float4>(), n_samples, c, rho_d, rat_d);
            CSL_LAUNCH_CHECK("tetrahedron densities");
            if (d == p->max_depth) break;
            d_split.ensure((size_t)nc * 4, s);
            k_dm_split<<<grid_for(nc, 256), 256, 0, s>>>(rho_d, tgt_d, nc, d_split.as<uint32_t>());
            CSL_LAUNCH_CHECK("split flags");
            const int64_t before = mesh.n_tets;
            const int64_t ns = mesh_subdivide(mesh, t0, nc, d_split.as<uint32_t>(), s);
            n_split += ns;
            per_tet(before, mesh.n_tets);
            t0 = before;
            nc = 8 * ns;
        }

        // the final edges (unsplit, in creation order) and the leaves
        MeshFinal fin;
        mesh_finalize(mesh, fin, s);
        const int64_t n_seg = fin.n_seg, n_leaf = fin.n_leaf;
        if (n_seg >= (1ll << 31)) fail(CSL_ERR_CAPACITY, "too many edges");

        // Step 3's per-edge minimum over the leaves containing the edge
        DevBuf d_r3((size_t)std::max<int64_t>(n_seg, 1) * 4, s);
        if (n_seg) {
            k_dm_fill_u32<<<grid_for(n_seg, 256), 256, 0, s>>>(d_r3.as<uint32_t>(), n_seg,
                                                               0x7f800000u);
            CSL_LAUNCH_CHECK("edge ratio start");
            mesh_edge_min(mesh, fin, d_ratio.as<float>(), d_r3.as<uint32_t>(), s);
            k_dm_ratio_fix<<<grid_for(n_seg, 256), 256, 0, s>>>(d_r3.as<uint32_t>(), n_seg);
            CSL_LAUNCH_CHECK("edge ratio default");
        }

        // Step 4: voxel-edge pairs, the per-voxel ratio, the per-edge minimum
        DevBuf d_sa((size_t)std::max<int64_t>(n_seg, 1) * 16, s),
            d_sb((size_t)std::max<int64_t>(n_seg, 1) * 16, s);
        mesh_segment_points(mesh, fin, d_sa.as<float4>(), d_sb.as<float4>(), s);
        const double reach = R * (1.0 + 1e-6) + 1e-6 * vox->h;
        DevBuf d_vr((size_t)n_vox * 4, s), d_rf((size_t)std::max<int64_t>(n_seg, 1) * 4, s);
        if (n_seg)
            CSL_CUDA(cudaMemcpyAsync(d_rf.get(), d_r3.get(), n_seg * 4, cudaMemcpyDeviceToDevice, s));
        int64_t n_pairs = 0;
        if (n_seg) {
            DevBuf d_cnt((size_t)n_seg * 4, s), d_off((size_t)n_seg * 8, s), d_tot(8, s);
            k_dm_vox_count<<<grid_for(n_seg, 256), 256, 0, s>>>(d_sa.as<float4>(), d_sb.as<float4>(),
                                                                n_seg, g, reach, d_cnt.as<uint32_t>());
            CSL_LAUNCH_CHECK("voxel pair count");
            exclusive_scan_u32_to_i64(d_cnt.as<uint32_t>(), d_off.as<int64_t>(), n_seg,
                                      d_tot.as<int64_t>(), s);
            n_pairs = read_i64(d_tot.as<int64_t>(), s);
            if (n_pairs >= (1ll << 31)) fail(CSL_ERR_CAPACITY, "more than 2^31 voxel-edge pairs");
            const size_t pb = (size_t)std::max<int64_t>(n_pairs, 1) * 4;
            DevBuf d_k(pb, s), d_v(pb, s), d_k2(pb, s), d_v2(pb, s);
            DevBuf d_vb((size_t)n_vox * 4, s), d_ve((size_t)n_vox * 4, s);
            CSL_CUDA(cudaMemsetAsync(d_vb.get(), 0, (size_t)n_vox * 4, s));
            CSL_CUDA(cudaMemsetAsync(d_ve.get(), 0, (size_t)n_vox * 4, s));
            if (n_pairs) {
                k_dm_vox_emit<<<grid_for(n_seg, 256), 256, 0, s>>>(
                    d_sa.as<float4>(), d_sb.as<float4>(), n_seg, g, reach, d_off.as<int64_t>(),
                    d_k.as<uint32_t>(), d_v.as<uint32_t>());
                CSL_LAUNCH_CHECK("voxel pair emit");
                int bits = 1;
                while (bits < 32 && (1ll << bits) < n_vox) ++bits;
                radix_sort_pairs(d_k.as<uint32_t>(), d_v.as<uint32_t>(), d_k2.as<uint32_t>(),
                                 d_v2.as<uint32_t>(), n_pairs, bits, s);
                k_dm_vox_bounds<<<grid_for(n_pairs, 256), 256, 0, s>>>(
                    d_k.as<uint32_t>(), n_pairs, d_vb.as<uint32_t>(), d_ve.as<uint32_t>());
                CSL_LAUNCH_CHECK("voxel pair bounds");
            }
            k_dm_voxel<<<(unsigned)std::min<int64_t>(n_vox, 152 * 5), kDmThreads, 0, s>>>(
                d_v.as<uint32_t>(), d_vb.as<uint32_t>(), d_ve.as<uint32_t>(), d_sa.as<float4>(),
                d_sb.as<float4>(), d_r3.as<float>(), d_tgt.as<float>(), g, c, p->vox_m,
                d_vr.as<float>());
            CSL_LAUNCH_CHECK("voxel ratios");
            if (n_pairs) {
                k_dm_vox_min<<<grid_for(n_pairs, 256), 256, 0, s>>>(
                    d_k.as<uint32_t>(), d_v.as<uint32_t>(), n_pairs, d_vr.as<float>(),
                    d_rf.as<uint32_t>());
                CSL_LAUNCH_CHECK("voxel ratio minimum");
            }
        } else {
            std::vector<uint32_t> nan(n_vox, 0x7fc00000u);
            CSL_CUDA(cudaMemcpyAsync(d_vr.get(), nan.data(), n_vox * 4, cudaMemcpyHostToDevice, s));
        }
        DevBuf d_rad((size_t)std::max<int64_t>(n_seg, 1) * 4, s);
        if (n_seg) {
            k_dm_radii<<<grid_for(n_seg, 256), 256, 0, s>>>(d_rf.as<float>(), n_seg, (float)r0,
                                                            d_rad.as<float>());
            CSL_LAUNCH_CHECK("radii");
        }
        std::vector<float> h_rad, h_r3, h_vr;
        download(h_rad, d_rad, n_seg, s);
        download(h_r3, d_r3, n_seg, s);
        download(h_vr, d_vr, n_vox, s);

        // the result, gathered on the device and copied into page-locked host blocks
        DevBuf g_edges((size_t)std::max<int64_t>(n_seg, 1) * 8, s),
            g_tets((size_t)std::max<int64_t>(n_leaf, 1) * 16, s),
            g_depth((size_t)std::max<int64_t>(n_leaf, 1) * 4, s),
            g_target((size_t)std::max<int64_t>(n_leaf, 1) * 8, s),
            g_rho((size_t)std::max<int64_t>(n_leaf, 1) * 4, s),
            g_ratio((size_t)std::max<int64_t>(n_leaf, 1) * 4, s);
        mesh_gather_final(mesh, fin, g_edges.as<int32_t>(), g_tets.as<int32_t>(),
                          g_depth.as<int32_t>(), d_target.as<double>(), g_target.as<double>(),
                          d_rho.as<float>(), g_rho.as<float>(), d_ratio.as<float>(),
                          g_ratio.as<float>(), s);
        host.start();
        csl_dm_result* r = (csl_dm_result*)calloc(1, sizeof(csl_dm_result));
        if (!r) fail(CSL_ERR_OOM, "result");
        auto to_block = [&](const DevBuf& b, size_t bytes) {
            void* h = host_block_alloc(bytes ? bytes : 16);
            if (!h) fail(CSL_ERR_OOM, "host result block");
            if (bytes) read_to_host(h, b.get(), bytes, s);
            return h;
        };
        r->n_nodes = mesh.n_nodes;
        r->nodes = (float*)to_block(mesh.xyz, (size_t)mesh.n_nodes * 12);
        r->n_edges = n_seg;
        r->edges = (int32_t*)to_block(g_edges, (size_t)n_seg * 8);
        r->radius = (float*)host_copy(h_rad.data(), h_rad.size() * 4);
        r->step3_ratio = (float*)host_copy(h_r3.data(), h_r3.size() * 4);
        r->n_tets = n_leaf;
        r->tets = (int32_t*)to_block(g_tets, (size_t)n_leaf * 16);
        r->tet_depth = (int32_t*)to_block(g_depth, (size_t)n_leaf * 4);
        r->tet_target = (double*)to_block(g_target, (size_t)n_leaf * 8);
        r->tet_rho_star = (float*)to_block(g_rho, (size_t)n_leaf * 4);
        r->tet_ratio = (float*)to_block(g_ratio, (size_t)n_leaf * 4);
        r->n_voxels = n_vox;
        r->voxel_ratio = (float*)host_copy(h_vr.data(), h_vr.size() * 4);
        r->n_subdivided = n_split;
        host.stop();
        wall.stop();
        r->host_ms = host.ms;
        r->wall_ms = wall.ms;
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

extern "C" void csl_dm_result_free(csl_dm_result* r) {
    if (!r) return;
    void* blocks[] = {r->nodes, r->edges, r->radius, r->step3_ratio, r->tets, r->tet_depth,
                      r->tet_target, r->tet_rho_star, r->tet_ratio, r->voxel_ratio};
    for (void* b : blocks)
        if (b) host_block_free(b);
    free(r);
}
