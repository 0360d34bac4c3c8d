// Ray casting of the implicit solid {Sigma >= C} into a headless depth image
// (the paper renders its lattices by ray tracing the implicit function,
// without a mesh; the field is that of Eq. 5-7).
//
// The struts are binned into a uniform 3D grid (each strut into every cell
// its support box meets: count, scan, emit, radix sort by cell). A ray is
// sampled at t_in + k * step from where it enters the lattice's box grown by
// R; Sigma at a sample sums the struts listed for the sample's cell (every
// strut whose support reaches the point is listed there); the first sample
// with Sigma >= C is refined by `refine` halvings of the last step. A cell
// with no strut has Sigma = 0 everywhere, so the ray jumps over it.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "field_tile.cuh"
#include "slice.cuh"

namespace csl {
namespace {

struct RvGrid {
    float lox, loy, loz, h;   // grid corner and cell edge
    int32_t nx, ny, nz;
};

struct RvConst {
    float ex, ey, ez;          // eye
    float fx, fy, fz;          // forward
    float rx, ry, rz;          // right
    float ux, uy, uz;          // up
    float half_w, half_h;      // image-plane half extents at distance 1
    int32_t width, height;
    float step;
    int32_t refine;
    float blo[3], bhi[3];      // the lattice's box grown by R
    float R2, inv_R4, C;
};

__device__ __forceinline__ bool strut_cells(const csl_rec& r, const RvGrid& g, float R, int& i0,
                                            int& i1, int& j0, int& j1, int& k0, int& k1) {
    const float bx = r.ax + r.len * r.ux, by = r.ay + r.len * r.uy, bz = r.az + r.len * r.uz;
    const float lo[3] = {fminf(r.ax, bx) - R, fminf(r.ay, by) - R, fminf(r.az, bz) - R};
    const float hi[3] = {fmaxf(r.ax, bx) + R, fmaxf(r.ay, by) + R, fmaxf(r.az, bz) + R};
    const float o[3] = {g.lox, g.loy, g.loz};
    const int n[3] = {g.nx, g.ny, g.nz};
    int a[3], b[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = max(0, min(n[k] - 1, (int)floorf((lo[k] - o[k]) / g.h)));
        b[k] = max(0, min(n[k] - 1, (int)floorf((hi[k] - o[k]) / g.h)));
    }
    i0 = a[0]; i1 = b[0]; j0 = a[1]; j1 = b[1]; k0 = a[2]; k1 = b[2];
    return true;
}

__global__ void k_rv_count(const csl_rec* __restrict__ rec, int64_t n, RvGrid g, float R,
                           uint32_t* __restrict__ cnt) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int i0, i1, j0, j1, k0, k1;
        strut_cells(rec[s], g, R, i0, i1, j0, j1, k0, k1);
        cnt[s] = (uint32_t)((i1 - i0 + 1) * (j1 - j0 + 1) * (k1 - k0 + 1));
    }
}

__global__ void k_rv_emit(const csl_rec* __restrict__ rec, int64_t n, RvGrid g, float R,
                          const int64_t* __restrict__ off, uint32_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int i0, i1, j0, j1, k0, k1;
        strut_cells(rec[s], g, R, i0, i1, j0, j1, k0, k1);
        int64_t o = off[s];
        for (int k = k0; k <= k1; ++k)
            for (int j = j0; j <= j1; ++j)
                for (int i = i0; i <= i1; ++i) {
                    keys[o] = (uint32_t)(((int64_t)k * g.ny + j) * g.nx + i);
                    vals[o] = (uint32_t)s;
                    ++o;
                }
    }
}

__global__ void k_rv_bounds(const uint32_t* __restrict__ keys, int64_t n,
                            uint32_t* __restrict__ beg, uint32_t* __restrict__ end) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) beg[k] = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) end[k] = (uint32_t)(i + 1);
    }
}

// Cell of a point, or -1 outside the grid.
__device__ __forceinline__ int64_t cell_of(float px, float py, float pz, const RvGrid& g,
                                           int& ci, int& cj, int& ck) {
    ci = (int)floorf((px - g.lox) / g.h);
    cj = (int)floorf((py - g.loy) / g.h);
    ck = (int)floorf((pz - g.loz) / g.h);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) return -1;
    return ((int64_t)ck * g.ny + cj) * g.nx + ci;
}

__device__ float sigma_at(float px, float py, float pz, const csl_rec* __restrict__ rec,
                          const uint32_t* __restrict__ vals, const uint32_t* __restrict__ cbeg,
                          const uint32_t* __restrict__ cend, const RvGrid& g, const RvConst& c) {
    int ci, cj, ck;
    const int64_t cell = cell_of(px, py, pz, g, ci, cj, ck);
    if (cell < 0) return 0.0f;
    float sig = 0.0f;
    for (uint32_t q = cbeg[cell]; q < cend[cell]; ++q) {
        const csl_rec r = rec[vals[q]];
        const float qx = px - r.ax, qy = py - r.ay, qz = pz - r.az;
        const float t0 = qx * r.ux + qy * r.uy + qz * r.uz;
        const float ex = qx - t0 * r.ux, ey = qy - t0 * r.uy, ez = qz - t0 * r.uz;
        const float h2 = c.R2 - (ex * ex + ey * ey + ez * ez);
        if (h2 > 0.0f && r.len > 0.0f) sig += (r.w * c.inv_R4) * segment_term_R4(t0, h2, r.len);
    }
    return sig;
}

// One thread per pixel: depth along its unit ray, +inf for a miss.
__global__ void k_rv_render(const csl_rec* __restrict__ rec, const uint32_t* __restrict__ vals,
                            const uint32_t* __restrict__ cbeg, const uint32_t* __restrict__ cend,
                            RvGrid g, RvConst c, float* __restrict__ depth) {
    const int64_t n_px = (int64_t)c.width * c.height;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_px;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % c.width), j = (int)(p / c.width);
        const float x = (((float)i + 0.5f) / (float)c.width * 2.0f - 1.0f) * c.half_w;
        const float y = (1.0f - ((float)j + 0.5f) / (float)c.height * 2.0f) * c.half_h;
        float dx = c.fx + x * c.rx + y * c.ux, dy = c.fy + x * c.ry + y * c.uy,
              dz = c.fz + x * c.rz + y * c.uz;
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv;
        dy *= inv;
        dz *= inv;
        const float o[3] = {c.ex, c.ey, c.ez}, d[3] = {dx, dy, dz};
        // the ray's interval in the box grown by R
        float t_in = 0.0f, t_out = INFINITY;
        bool miss = false;
        for (int k = 0; k < 3 && !miss; ++k) {
            if (d[k] == 0.0f) {
                miss = o[k] < c.blo[k] || o[k] > c.bhi[k];
                continue;
            }
            float a = (c.blo[k] - o[k]) / d[k], b = (c.bhi[k] - o[k]) / d[k];
            if (a > b) {
                const float t = a;
                a = b;
                b = t;
            }
            t_in = fmaxf(t_in, a);
            t_out = fminf(t_out, b);
            miss = t_in > t_out;
        }
        float result = INFINITY;
        if (!miss) {
            const int64_t k_max = (int64_t)floorf((t_out - t_in) / c.step);
            for (int64_t k = 0; k <= k_max;) {
                const float t = t_in + c.step * (float)k;
                const float px = o[0] + t * d[0], py = o[1] + t * d[1], pz = o[2] + t * d[2];
                int ci, cj, ck;
                const int64_t cell = cell_of(px, py, pz, g, ci, cj, ck);
                if (cell >= 0 && cbeg[cell] == cend[cell]) {
                    // an empty cell: jump to the first sample past it
                    float t_exit = INFINITY;
                    const int cc[3] = {ci, cj, ck};
                    const float lo3[3] = {g.lox, g.loy, g.loz};
                    for (int a = 0; a < 3; ++a) {
                        if (d[a] == 0.0f) continue;
                        const float bound = lo3[a] + g.h * (float)(d[a] > 0.0f ? cc[a] + 1 : cc[a]);
                        t_exit = fminf(t_exit, (bound - o[a]) / d[a]);
                    }
                    const int64_t kn = (int64_t)floorf((t_exit - t_in) / c.step) + 1;
                    k = kn > k ? kn : k + 1;
                    continue;
                }
                const float s = cell < 0 ? 0.0f : sigma_at(px, py, pz, rec, vals, cbeg, cend, g, c);
                if (s >= c.C) {
                    if (k == 0) {
                        result = t_in;
                    } else {
                        float lo = t_in + c.step * (float)(k - 1), hi = t;
                        for (int it = 0; it < c.refine; ++it) {
                            const float m = 0.5f * (lo + hi);
                            const float sm = sigma_at(o[0] + m * d[0], o[1] + m * d[1],
                                                      o[2] + m * d[2], rec, vals, cbeg, cend, g, c);
                            if (sm >= c.C)
                                hi = m;
                            else
                                lo = m;
                        }
                        result = 0.5f * (lo + hi);
                    }
                    break;
                }
                ++k;
            }
        }
        depth[p] = result;
    }
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" csl_status csl_render_depth(const csl_lattice* L, const csl_camera* cam, float* depth,
                                       void* stream) {
    try {
        if (!L || !cam || !depth) fail(CSL_ERR_INVALID_ARG, "NULL argument");
        require_device_resident(L);
        if (cam->width < 1 || cam->height < 1 || (int64_t)cam->width * cam->height >= (1ll << 31))
            fail(CSL_ERR_INVALID_ARG, "width and height must be >= 1");
        if (!(cam->fov_y > 0.0 && cam->fov_y < M_PI)) fail(CSL_ERR_INVALID_ARG, "fov_y in (0, pi)");
        if (!(cam->step > 0.0) || !isfinite(cam->step)) fail(CSL_ERR_INVALID_ARG, "step must be > 0");
        if (cam->refine < 0 || cam->refine > 60) fail(CSL_ERR_INVALID_ARG, "refine in [0, 60]");
        double f[3], up[3], r[3], u[3];
        for (int k = 0; k < 3; ++k) {
            if (!isfinite(cam->eye[k]) || !isfinite(cam->target[k]) || !isfinite(cam->up[k]))
                fail(CSL_ERR_INVALID_ARG, "non-finite camera");
            f[k] = cam->target[k] - cam->eye[k];
            up[k] = cam->up[k];
        }
        const double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        if (!(fn > 0.0)) fail(CSL_ERR_INVALID_ARG, "target equals eye");
        for (int k = 0; k < 3; ++k) f[k] /= fn;
        r[0] = f[1] * up[2] - f[2] * up[1];
        r[1] = f[2] * up[0] - f[0] * up[2];
        r[2] = f[0] * up[1] - f[1] * up[0];
        const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (!(rn > 0.0)) fail(CSL_ERR_INVALID_ARG, "up is parallel to the view direction");
        for (int k = 0; k < 3; ++k) r[k] /= rn;
        u[0] = r[1] * f[2] - r[2] * f[1];
        u[1] = r[2] * f[0] - r[0] * f[2];
        u[2] = r[0] * f[1] - r[1] * f[0];
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n_px = (int64_t)cam->width * cam->height;
        const int64_t ne = L->n_edges;
        const double R = L->R;
        RvConst c;
        c.ex = (float)cam->eye[0];
        c.ey = (float)cam->eye[1];
        c.ez = (float)cam->eye[2];
        c.fx = (float)f[0]; c.fy = (float)f[1]; c.fz = (float)f[2];
        c.rx = (float)r[0]; c.ry = (float)r[1]; c.rz = (float)r[2];
        c.ux = (float)u[0]; c.uy = (float)u[1]; c.uz = (float)u[2];
        c.half_h = (float)tan(0.5 * cam->fov_y);
        c.half_w = (float)(tan(0.5 * cam->fov_y) * cam->width / cam->height);
        c.width = cam->width;
        c.height = cam->height;
        c.step = (float)cam->step;
        c.refine = cam->refine;
        for (int k = 0; k < 3; ++k) {
            c.blo[k] = (float)((double)L->bbox_lo[k] - R);
            c.bhi[k] = (float)((double)L->bbox_hi[k] + R);
        }
        c.R2 = (float)(R * R);
        c.inv_R4 = (float)(1.0 / (R * R * R * R));
        c.C = (float)L->C;
        if (ne == 0) {
            // no struts: every ray misses
            std::vector<float> inf(n_px, INFINITY);
            CSL_CUDA(cudaMemcpyAsync(depth, inf.data(), n_px * 4, cudaMemcpyHostToDevice, s));
            CSL_CUDA(cudaStreamSynchronize(s));
            return CSL_OK;
        }
        // at most 2^24 samples along any ray through the box, so that the
        // sample index k is exact in float and every march ends in bounded time
        {
            double diag2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double e = (double)c.bhi[k] - (double)c.blo[k];
                diag2 += e * e;
            }
            if (sqrt(diag2) / cam->step > (double)(1 << 24))
                fail(CSL_ERR_INVALID_ARG, "step too small: more than 2^24 samples across the box");
        }
        // the grid: cells of edge >= 2R, at most 2^24 of them
        RvGrid g;
        double h = std::max(2.0 * R, 1e-6);
        auto dims_of = [&](double hh, int* d) {
            int64_t tot = 1;
            for (int k = 0; k < 3; ++k) {
                d[k] = (int)std::max<double>(1.0, ceil((double)(c.bhi[k] - c.blo[k]) / hh) + 1.0);
                tot *= d[k];
            }
            return tot;
        };
        int dims[3];
        while (dims_of(h, dims) > (1ll << 24)) h *= 1.25;
        g.lox = c.blo[0];
        g.loy = c.blo[1];
        g.loz = c.blo[2];
        g.h = (float)h;
        g.nx = dims[0];
        g.ny = dims[1];
        g.nz = dims[2];
        const int64_t n_cells = (int64_t)g.nx * g.ny * g.nz;
        const csl_rec* rec = L->rec.as<csl_rec>();
        DevBuf d_cnt((size_t)ne * 4, s), d_off((size_t)ne * 8, s), d_tot(8, s);
        k_rv_count<<<grid_for(ne, 256), 256, 0, s>>>(rec, ne, g, (float)R, d_cnt.as<uint32_t>());
        CSL_LAUNCH_CHECK("render cell counts");
        exclusive_scan_u32_to_i64(d_cnt.as<uint32_t>(), d_off.as<int64_t>(), ne, d_tot.as<int64_t>(), s);
        const int64_t n_pairs = read_i64(d_tot.as<int64_t>(), s);
        if (n_pairs >= (1ll << 31)) fail(CSL_ERR_CAPACITY, "more than 2^31 strut-cell pairs");
        const size_t pb = (size_t)std::max<int64_t>(n_pairs, 1) * 4;
        DevBuf d_k(pb, s), d_v(pb, s), d_k2(pb, s), d_v2(pb, s);
        DevBuf d_cb((size_t)n_cells * 4, s), d_ce((size_t)n_cells * 4, s);
        CSL_CUDA(cudaMemsetAsync(d_cb.get(), 0, (size_t)n_cells * 4, s));
        CSL_CUDA(cudaMemsetAsync(d_ce.get(), 0, (size_t)n_cells * 4, s));
        k_rv_emit<<<grid_for(ne, 256), 256, 0, s>>>(rec, ne, g, (float)R, d_off.as<int64_t>(),
                                                    d_k.as<uint32_t>(), d_v.as<uint32_t>());
        CSL_LAUNCH_CHECK("render cell pairs");
        int bits = 1;
        while (bits < 32 && (1ll << bits) < n_cells) ++bits;
        radix_sort_pairs(d_k.as<uint32_t>(), d_v.as<uint32_t>(), d_k2.as<uint32_t>(),
                         d_v2.as<uint32_t>(), n_pairs, bits, s);
        k_rv_bounds<<<grid_for(n_pairs, 256), 256, 0, s>>>(d_k.as<uint32_t>(), n_pairs,
                                                           d_cb.as<uint32_t>(), d_ce.as<uint32_t>());
        CSL_LAUNCH_CHECK("render cell bounds");
        k_rv_render<<<grid_for(n_px, 128), 128, 0, s>>>(rec, d_v.as<uint32_t>(), d_cb.as<uint32_t>(),
                                                        d_ce.as<uint32_t>(), g, c, depth);
        CSL_LAUNCH_CHECK("render rays");
        CSL_CUDA(cudaStreamSynchronize(s));
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
