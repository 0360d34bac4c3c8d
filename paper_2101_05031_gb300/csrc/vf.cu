// Smoothed volume fraction per density cell (Eq. 9, read with stratified
// samples and a sigmoid) and its adjoint with respect to the strut radii and
// the node positions (the radius tuning of Sec. 5.4).
//
//   vf_c = (1/m^3) sum_k sigmoid((Sigma(p_ck) - C) / T),
//   p_ck = o + h (c + (k + 1/2) / m) per axis.
//
// The m^3 samples of every cell are the pixels of a grid of pixel size h/m and
// the cell layers are slabs of S = m layers, so the forward pass reuses the
// slab/tile binner and the field kernel; a warp per cell then averages the
// sigmoid. The backward pass is one kernel per (tile, slab): pass 1 recomputes
// Sigma at its samples (nothing is stored between forward and backward) and
// turns it into alpha = g_c / m^3 * s (1 - s) / T; pass 2 evaluates, for every
// staged edge, the derivatives of its segment integral with respect to the
// edge's weight and endpoints, sums them over the CTA's samples (per thread,
// then a fixed warp tree, then the warps in order) and writes one partial per
// bin entry. The partials are summed per edge in a fixed order (stable sort by
// edge), and node gradients are gathered through a node -> endpoint list, so
// the result is deterministic.
//
// Derivatives of I = int_0^L f(|p - a - t u|^2) dt (f quartic, Eq. 5) by
// differentiating under the integral in the fixed-bounds form
// L int_0^1 f(|p - a - s (b - a)|^2) ds (f and f' vanish on the support
// sphere, so the moving clip points add nothing). With p - a = t0 u + e and the
// moments M_k = int (h2 - tau^2) tau^k dtau over the clipped interval:
//   R^4 dI/da = -u R^4 I / L - 4 [u ((1 - t0/L) M1 - M2/L) - e ((1 - t0/L) M0 - M1/L)]
//   R^4 dI/db = +u R^4 I / L - 4 [u ((t0/L) M1 + M2/L) - e ((t0/L) M0 + M1/L)]
// The integrands are polynomials of degree <= 4 in tau, so the same 3-point
// Gauss-Legendre rule gives I and the three moments exactly.
#include <math.h>

#include <algorithm>
#include <vector>

#include "field_tile.cuh"
#include "slice.cuh"

namespace csl {
namespace {

constexpr int kVfThreads = 256;

ChunkGeom vf_geom(const csl_lattice* L, const csl_cells& cells, int first_cl, int n_cl) {
    const int m = cells.m;
    ChunkGeom g;
    g.nx = cells.dims[0] * m;
    g.ny = cells.dims[1] * m;
    g.ntx = (g.nx + kTile - 1) / kTile;
    g.nty = (g.ny + kTile - 1) / kTile;
    g.px = cells.h / m;
    g.x0 = cells.origin[0];
    g.y0 = cells.origin[1];
    g.dz = cells.h / m;
    g.z0 = cells.origin[2] + 0.5 * g.dz;
    g.first_layer = first_cl * m;
    g.n_layers = n_cl * m;
    g.S = m;
    g.n_slabs = n_cl;
    g.R = L->R;
    double scale = 1.0;
    for (int k = 0; k < 3; ++k)
        scale = std::max({scale, fabs((double)L->bbox_lo[k]), fabs((double)L->bbox_hi[k]),
                          fabs(cells.origin[k]), fabs(cells.origin[k] + cells.dims[k] * cells.h)});
    g.margin_xy = g.margin_z = (float)(L->R + 8e-6 * scale + 1e-6);
    return g;
}

void validate_cells(const csl_cells* c) {
    if (!c) fail(CSL_ERR_INVALID_ARG, "cells is NULL");
    if (!(c->m == 1 || c->m == 2 || c->m == 4 || c->m == 8))
        fail(CSL_ERR_INVALID_ARG, "samples per cell axis m must be 1, 2, 4 or 8");
    for (int k = 0; k < 3; ++k) {
        if (c->dims[k] < 1) fail(CSL_ERR_INVALID_ARG, "cell dims must be >= 1");
        if (!isfinite(c->origin[k])) fail(CSL_ERR_INVALID_ARG, "non-finite cell origin");
    }
    if ((int64_t)c->dims[0] * c->m > 32000 || (int64_t)c->dims[1] * c->m > 32000)
        fail(CSL_ERR_INVALID_ARG, "dims[0] * m and dims[1] * m must be <= 32000");
    if ((int64_t)c->dims[2] * c->m > 65535)
        fail(CSL_ERR_INVALID_ARG, "dims[2] * m must be <= 65535");
    if (!(isfinite(c->h) && c->h > 0)) fail(CSL_ERR_INVALID_ARG, "cell size h must be > 0");
    if (!(isfinite(c->temperature) && c->temperature > 0))
        fail(CSL_ERR_INVALID_ARG, "temperature must be > 0");
}

// cell layers per chunk: about 1 GiB of Sigma, at least one
int vf_chunk_cell_layers(const csl_cells& c) {
    const int64_t per_cl = (int64_t)c.dims[0] * c.dims[1] * c.m * c.m * c.m * 4;
    int64_t n = ((int64_t)1 << 30) / std::max<int64_t>(per_cl, 1);
    n = std::max<int64_t>(1, std::min<int64_t>(n, c.dims[2]));
    // the binner keys (slab, tile) in 32 bits
    const int64_t tiles = ceil_div((int64_t)c.dims[0] * c.m, kTile) * ceil_div((int64_t)c.dims[1] * c.m, kTile);
    n = std::min<int64_t>(n, std::max<int64_t>(1, 0xffffffffLL / std::max<int64_t>(tiles, 1)));
    return (int)n;
}

__device__ __forceinline__ float sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }

// one warp per cell of the chunk
__global__ void k_vf_mean(const float* __restrict__ sigma, int cx, int cy, int n_cl, int m, float C,
                          float invT, float* __restrict__ vf) {
    const int lane = threadIdx.x & 31;
    const int64_t n_cells = (int64_t)cx * cy * n_cl;
    const int64_t nx = (int64_t)cx * m, ny = (int64_t)cy * m;
    const int m3 = m * m * m;
    for (int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; cell < n_cells;
         cell += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int ix = (int)(cell % cx), iy = (int)((cell / cx) % cy), iz = (int)(cell / ((int64_t)cx * cy));
        float acc = 0.0f;
        for (int s = lane; s < m3; s += 32) {
            const int kx = s % m, ky = (s / m) % m, kz = s / (m * m);
            const int64_t i = (int64_t)ix * m + kx, j = (int64_t)iy * m + ky;
            const int64_t l = (int64_t)iz * m + kz;
            acc += sigmoid((sigma[(l * ny + j) * nx + i] - C) * invT);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) vf[cell] = acc / (float)m3;
    }
}

struct GradConst {
    int32_t nx, ny, ntx, n_tiles, n_layers;
    int32_t cx, cy, m, first_cl;
    float R2, fpx, fdz, C, invT, inv_m3;
    float span_r2;   // squared radius of the footprint rows (R plus slack)
    TileCull tc;
    const float2* org_x;
    const float2* org_y;
    const float2* org_z;
};

// Per (tile, slab): pass 1 Sigma -> alpha; pass 2 partial derivatives per
// staged edge. partial[entry] = {sum alpha R^4 I, sum alpha w dI/da (3),
// sum alpha w dI/db (3), 0}.
template <int S>
__global__ void __launch_bounds__(kVfThreads, 6)
k_vf_grad(const csl_rec* __restrict__ rec, const uint32_t* __restrict__ vals,
          const uint32_t* __restrict__ tstart, const uint32_t* __restrict__ tend, GradConst c,
          const float* __restrict__ g_cells, float4* __restrict__ partial) {
    __shared__ float4 s_a[kVfThreads];
    __shared__ float4 s_b[kVfThreads];
    __shared__ uint64_t s_mask[kVfThreads];
    __shared__ float s_alpha[S * kTile * kTile];   // [layer][j][i]

    const int tile = blockIdx.x, slab = blockIdx.y;
    const int tx = tile % c.ntx, ty = tile / c.ntx;
    const uint32_t key = (uint32_t)slab * (uint32_t)c.n_tiles + (uint32_t)tile;
    const uint32_t beg = tstart[key], end = tend[key];
    if (end <= beg) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    (void)lane;
    const int wx = warp & 1, wy = warp >> 1;
    const int il = wx * 8 + (lane & 7), jl = wy * 4 + (lane >> 3);
    const int l0 = slab * S;
    const int nl = min(S, c.n_layers - l0);
    const float2 ox = c.org_x[tx], oy = c.org_y[ty], oz = c.org_z[slab];
    const float pxl = ((float)il + 0.5f) * c.fpx, pyl = ((float)jl + 0.5f) * c.fpx;
    const TileCull cull = c.tc;

    // pass 1: Sigma at this thread's samples
    float acc[S];
#pragma unroll
    for (int l = 0; l < S; ++l) acc[l] = 0.0f;
    for (uint32_t c0 = beg; c0 < end; c0 += kVfThreads) {
        const int cnt = (int)min((uint32_t)kVfThreads, end - c0);
        if ((int)threadIdx.x < cnt) {
            float4 A, B;
            s_mask[threadIdx.x] = stage_record(rec + vals[c0 + threadIdx.x], ox.x, ox.y, oy.x,
                                               oy.y, oz.x, oz.y, nl, cull, A, B);
            s_a[threadIdx.x] = A;
            s_b[threadIdx.x] = B;
        }
        __syncthreads();
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const uint32_t wm = i < cnt ? (uint32_t)(s_mask[i] >> (warp * 8)) & 0xffu : 0u;
            uint32_t ball = __ballot_sync(0xffffffffu, wm != 0u);
            while (ball) {
                const int b = __ffs(ball) - 1;
                ball &= ball - 1u;
                const uint32_t lm = __shfl_sync(0xffffffffu, wm, b);
                const float4 A = s_a[i0 + b], B = s_b[i0 + b];
                const float dx = pxl - A.x, dy = pyl - A.y;
                const float txy = fmaf(dy, B.x, dx * A.w);
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    if (lm & (1u << l)) {
                        const float dz = (float)l * c.fdz - A.z;
                        const float t0 = fmaf(dz, B.y, txy);
                        const float ex = fmaf(-t0, A.w, dx), ey = fmaf(-t0, B.x, dy);
                        const float ez = fmaf(-t0, B.y, dz);
                        const float h2 = fmaxf(c.R2 - fmaf(ez, ez, fmaf(ey, ey, ex * ex)), 0.0f);
                        acc[l] = fmaf(B.w, segment_term_R4(t0, h2, B.z), acc[l]);
                    }
                }
            }
        }
        __syncthreads();
    }
    // alpha = dL/dSigma at each sample
    const int gi = tx * kTile + il, gj = ty * kTile + jl;
    float alpha[S];
#pragma unroll
    for (int l = 0; l < S; ++l) {
        alpha[l] = 0.0f;
        if (l < nl && gi < c.nx && gj < c.ny) {
            const int lz = l0 + l;   // chunk-local sample layer
            const int64_t cell =
                ((int64_t)(c.first_cl + lz / c.m) * c.cy + gj / c.m) * c.cx + gi / c.m;
            const float s = sigmoid((acc[l] - c.C) * c.invT);
            alpha[l] = g_cells[cell] * c.inv_m3 * s * (1.0f - s) * c.invT;
        }
    }
    // alpha of every sample of the tile, for pass 2 (0 outside the grid / slab)
#pragma unroll
    for (int l = 0; l < S; ++l) s_alpha[(l * kTile + jl) * kTile + il] = alpha[l];
    // pass 2: one staged edge per thread; the thread visits the samples of its
    // edge's footprint (rows of the clipped box, cut to the pixels within R of
    // the line) and sums the 7 partials in registers, in a fixed order. A
    // sample with alpha == 0 (the sigmoid saturates to 0 or 1 in FP32) adds
    // exactly nothing and is skipped.
    for (uint32_t c0 = beg; c0 < end; c0 += kVfThreads) {
        const int cnt = (int)min((uint32_t)kVfThreads, end - c0);
        __syncthreads();   // s_alpha written (first chunk) / nothing else shared here
        if ((int)threadIdx.x >= cnt) continue;
        float4 A, B;
        load_record(rec + vals[c0 + threadIdx.x], ox.x, ox.y, oy.x, oy.y, oz.x, oz.y,
                    cull.inv_R4, A, B);
        const float ux = A.w, uy = B.x, uz = B.y, len = B.z;
        const float inv_len = len > 0.0f ? 1.0f / len : 0.0f;
        float gw = 0.0f, gax = 0.0f, gay = 0.0f, gaz = 0.0f, gbx = 0.0f, gby = 0.0f, gbz = 0.0f;
        for (int l = 0; l < nl; ++l) {
            const uint32_t e = item_extent(A, B, l, cull);
            if (!e) continue;
            const float zl = (float)l * c.fdz;
            const int j0 = (int)(e & 15u), j1 = (int)((e >> 4) & 15u);
            for (int j = j0; j <= j1; ++j) {
                int i0, i1;
                if (!row_span(A, B, zl, j, e, cull, c.span_r2, i0, i1)) continue;
                const float dy = ((float)j + 0.5f) * c.fpx - A.y;
                const float dz = zl - A.z;
                const float* arow = s_alpha + (l * kTile + j) * kTile;
                for (int i = i0; i <= i1; ++i) {
                    const float al = arow[i];
                    if (al == 0.0f) continue;
                    const float dx = ((float)i + 0.5f) * c.fpx - A.x;
                    const float txy = fmaf(dy, uy, dx * ux);
                    const float t0 = fmaf(dz, uz, txy);
                    const float ex = fmaf(-t0, ux, dx), ey = fmaf(-t0, uy, dy);
                    const float ez = fmaf(-t0, uz, dz);
                    const float h2 = fmaxf(c.R2 - fmaf(ez, ez, fmaf(ey, ey, ex * ex)), 0.0f);
                    if (h2 == 0.0f) continue;
                    const float w = sqrt_approx(h2);
                    const float tau1 = fmaxf(-t0, -w), tau2 = fminf(len - t0, w);
                    const float hh = 0.5f * fmaxf(tau2 - tau1, 0.0f);   // half width
                    const float mm = 0.5f * (tau2 + tau1);               // midpoint
                    const float del = 0.7745966692414834f * hh;          // sqrt(0.6) h
                    const float ta = mm - del, tb = mm + del;
                    const float ga = fmaf(-ta, ta, h2), gm = fmaf(-mm, mm, h2),
                                gb = fmaf(-tb, tb, h2);
                    const float W1 = (5.0f / 9.0f) * hh, W2 = (8.0f / 9.0f) * hh;
                    const float wa = W1 * ga, wm2 = W2 * gm, wb = W1 * gb;
                    const float I4 = fmaf(wa, ga, fmaf(wm2, gm, wb * gb));
                    const float M0 = wa + wm2 + wb;
                    const float M1 = fmaf(wa, ta, fmaf(wm2, mm, wb * tb));
                    const float M2 = fmaf(wa * ta, ta, fmaf(wm2 * mm, mm, wb * tb * tb));
                    const float r = t0 * inv_len;
                    const float il4 = I4 * inv_len;
                    const float cau = fmaf(1.0f - r, M1, -M2 * inv_len);
                    const float cae = fmaf(1.0f - r, M0, -M1 * inv_len);
                    const float cbu = fmaf(r, M1, M2 * inv_len);
                    const float cbe = fmaf(r, M0, M1 * inv_len);
                    const float alw = al * B.w;
                    gw = fmaf(al, I4, gw);
                    // R^4 dI/da = -u I4/L - 4 (u cau - e cae); times alpha w/R^4
                    gax = fmaf(alw, fmaf(-ux, il4, -4.0f * fmaf(ux, cau, -ex * cae)), gax);
                    gay = fmaf(alw, fmaf(-uy, il4, -4.0f * fmaf(uy, cau, -ey * cae)), gay);
                    gaz = fmaf(alw, fmaf(-uz, il4, -4.0f * fmaf(uz, cau, -ez * cae)), gaz);
                    gbx = fmaf(alw, fmaf(ux, il4, -4.0f * fmaf(ux, cbu, -ex * cbe)), gbx);
                    gby = fmaf(alw, fmaf(uy, il4, -4.0f * fmaf(uy, cbu, -ey * cbe)), gby);
                    gbz = fmaf(alw, fmaf(uz, il4, -4.0f * fmaf(uz, cbu, -ez * cbe)), gbz);
                }
            }
        }
        partial[2 * (int64_t)(c0 + threadIdx.x)] = make_float4(gw, gax, gay, gaz);
        partial[2 * (int64_t)(c0 + threadIdx.x) + 1] = make_float4(gbx, gby, gbz, 0.0f);
    }
}

__global__ void k_iota(uint32_t* a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

// keys sorted by edge record, vals = entry index: per run of equal keys, the
// partials summed in entry order and added to acc[record] (7 floats, pitch 8).
__global__ void k_seg_sum(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                          int64_t n, const float4* __restrict__ partial, float* __restrict__ acc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i > 0 && keys[i - 1] == k) continue;
        float v[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t j = i; j < n && keys[j] == k; ++j) {
            const float4 a = partial[2 * (int64_t)vals[j]], b = partial[2 * (int64_t)vals[j] + 1];
            v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w;
            v[4] += b.x; v[5] += b.y; v[6] += b.z;
        }
        float* o = acc + 8 * (int64_t)k;
        for (int q = 0; q < 7; ++q) o[q] += v[q];
    }
}

// per record: dL/drho of its edge, and the gradients of its two endpoints
__global__ void k_edge_out(const float* __restrict__ acc, const uint32_t* __restrict__ sid,
                           const float* __restrict__ radius, int64_t n_edges, double R, double C,
                           int mode, float inv_R4, float* __restrict__ grad_radius,
                           float* __restrict__ gend) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_edges;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = sid[k] & 0x7fffffffu;
        const float* a = acc + 8 * k;
        const double rho = radius[j];
        double dw = 1.0;
        if (mode != CSL_MODE_RAW) {
            const double q = R * R - rho * rho;
            const double w = C * 15.0 * (R * R) * (R * R) / (16.0 * q * q * sqrt(q));
            dw = w * 5.0 * rho / q;
        }
        grad_radius[j] = (float)((double)a[0] * inv_R4 * dw);
        for (int q = 0; q < 6; ++q) gend[6 * k + q] = a[1 + q];
    }
}

// node -> endpoint list: keys = node id, vals = record << 1 | end (0: v_s)
__global__ void k_node_keys(const int32_t* __restrict__ edges, const uint32_t* __restrict__ sid,
                            int64_t n_edges, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals, uint32_t* __restrict__ count) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_edges;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = sid[k] & 0x7fffffffu;
        const bool swap = (sid[k] >> 31) != 0;
        const uint32_t lo = (uint32_t)edges[2 * (int64_t)j + (swap ? 1 : 0)];
        const uint32_t hi = (uint32_t)edges[2 * (int64_t)j + (swap ? 0 : 1)];
        keys[2 * k] = lo;
        vals[2 * k] = (uint32_t)(k << 1);
        keys[2 * k + 1] = hi;
        vals[2 * k + 1] = (uint32_t)(k << 1) | 1u;
        atomicAdd(&count[lo], 1u);
        atomicAdd(&count[hi], 1u);
    }
}

__global__ void k_node_grad(const int64_t* __restrict__ off, const uint32_t* __restrict__ ent,
                            const float* __restrict__ gend, int64_t n_nodes,
                            float* __restrict__ grad_nodes) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes;
         i += (int64_t)gridDim.x * blockDim.x) {
        float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            const uint32_t v = ent[e];
            const float* p = gend + 6 * (int64_t)(v >> 1) + 3 * (v & 1u);
            g0 += p[0];
            g1 += p[1];
            g2 += p[2];
        }
        grad_nodes[3 * i] = g0;
        grad_nodes[3 * i + 1] = g1;
        grad_nodes[3 * i + 2] = g2;
    }
}

int bits_for(int64_t n) {
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) < n) ++b;
    return b;
}

void build_node_csr(csl_lattice* L, cudaStream_t s) {
    const int64_t ne = L->n_edges, nn = L->n_nodes;
    L->node_csr_off.ensure_persistent((size_t)(nn + 1) * 8);
    L->node_csr.ensure_persistent((size_t)std::max<int64_t>(2 * ne, 1) * 4);
    DevBuf count((size_t)std::max<int64_t>(nn, 1) * 4, s);
    CSL_CUDA(cudaMemsetAsync(count.get(), 0, (size_t)std::max<int64_t>(nn, 1) * 4, s));
    if (ne > 0) {
        DevBuf keys(2 * ne * 4, s), tk(2 * ne * 4, s), tv(2 * ne * 4, s);
        k_node_keys<<<grid_for(ne, 256), 256, 0, s>>>(L->edges.as<int32_t>(), L->sid.as<uint32_t>(),
                                                     ne, keys.as<uint32_t>(),
                                                     L->node_csr.as<uint32_t>(), count.as<uint32_t>());
        CSL_LAUNCH_CHECK("node keys");
        radix_sort_pairs(keys.as<uint32_t>(), L->node_csr.as<uint32_t>(), tk.as<uint32_t>(),
                         tv.as<uint32_t>(), 2 * ne, bits_for(nn), s);
    }
    exclusive_scan_u32_to_i64(count.as<uint32_t>(), L->node_csr_off.as<int64_t>(), nn,
                              L->node_csr_off.as<int64_t>() + nn, s);
}

// uploads the tile / slab origins of a chunk as (hi, lo) float pairs
DevBuf origin_tables(const ChunkGeom& g, cudaStream_t s) {
    std::vector<float2> org((size_t)g.ntx + g.nty + g.n_slabs);
    auto split = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    for (int i = 0; i < g.ntx; ++i) org[i] = split(g.x0 + (double)(i * kTile) * g.px);
    for (int j = 0; j < g.nty; ++j) org[g.ntx + j] = split(g.y0 + (double)(j * kTile) * g.px);
    for (int k = 0; k < g.n_slabs; ++k)
        org[g.ntx + g.nty + k] = split(g.z0 + (double)(g.first_layer + k * g.S) * g.dz);
    DevBuf d(org.size() * sizeof(float2), s);
    CSL_CUDA(cudaMemcpyAsync(d.get(), org.data(), org.size() * sizeof(float2),
                             cudaMemcpyHostToDevice, s));
    return d;
}

TileCull tile_cull(const ChunkGeom& g) {
    TileCull t;
    t.fpx = (float)g.px;
    t.fdz = (float)g.dz;
    t.cull = (float)(g.R * (1.0 + 1e-5) + 1e-6);
    const double hd = g.px * sqrt(3.5 * 3.5 + 1.5 * 1.5) * (1.0 + 1e-5);
    const double r = (double)t.cull + hd;
    t.cull_line2 = (float)(r * r);
    t.inv_R4 = (float)(1.0 / (g.R * g.R * g.R * g.R));
    return t;
}

}  // namespace

void validate_cells_or_fail(const csl_cells* c) { validate_cells(c); }

void vf_forward(const csl_lattice* L, const csl_cells& cells, float* vf, cudaStream_t s) {
    const int per = vf_chunk_cell_layers(cells);
    const int cz = cells.dims[2];
    DevBuf sigma((size_t)cells.dims[0] * cells.dims[1] * per * cells.m * cells.m * cells.m * 4, s);
    for (int first = 0; first < cz; first += per) {
        const int n = std::min(per, cz - first);
        ChunkGeom g = vf_geom(L, cells, first, n);
        SlabBins bins;
        bin_chunk(L, g, bins, s);
        field_chunk(L, g, bins, (float)L->C, sigma.as<float>(), nullptr, nullptr, s);
        const int64_t n_cells = (int64_t)cells.dims[0] * cells.dims[1] * n;
        k_vf_mean<<<grid_for(n_cells * 32, 256), 256, 0, s>>>(
            sigma.as<float>(), cells.dims[0], cells.dims[1], n, cells.m, (float)L->C,
            (float)(1.0 / cells.temperature),
            vf + (int64_t)first * cells.dims[0] * cells.dims[1]);
        CSL_LAUNCH_CHECK("vf mean");
    }
}

void vf_backward(csl_lattice* L, const csl_cells& cells, const float* grad_vf, float* grad_radius,
                 float* grad_nodes, cudaStream_t s) {
    const int64_t ne = L->n_edges, nn = L->n_nodes;
    if (nn > 0) CSL_CUDA(cudaMemsetAsync(grad_nodes, 0, (size_t)nn * 12, s));
    if (ne == 0) return;
    const int per = vf_chunk_cell_layers(cells);
    const int cz = cells.dims[2];
    DevBuf acc((size_t)ne * 32, s);
    CSL_CUDA(cudaMemsetAsync(acc.get(), 0, (size_t)ne * 32, s));
    for (int first = 0; first < cz; first += per) {
        const int n = std::min(per, cz - first);
        ChunkGeom g = vf_geom(L, cells, first, n);
        SlabBins bins;
        bin_chunk(L, g, bins, s);
        if (bins.n_pairs == 0) continue;
        DevBuf partial((size_t)bins.n_pairs * 32, s);
        DevBuf org = origin_tables(g, s);
        GradConst c;
        c.nx = g.nx;
        c.ny = g.ny;
        c.ntx = g.ntx;
        c.n_tiles = g.ntx * g.nty;
        c.n_layers = g.n_layers;
        c.cx = cells.dims[0];
        c.cy = cells.dims[1];
        c.m = cells.m;
        c.first_cl = first;
        c.R2 = (float)(L->R * L->R);
        c.fpx = (float)g.px;
        c.fdz = (float)g.dz;
        c.C = (float)L->C;
        c.invT = (float)(1.0 / cells.temperature);
        c.inv_m3 = 1.0f / (float)(cells.m * cells.m * cells.m);
        c.tc = tile_cull(g);
        {
            const double rs = L->R * (1.0 + 2e-4) + 1e-6;
            c.span_r2 = (float)(rs * rs);
        }
        c.org_x = org.as<float2>();
        c.org_y = c.org_x + g.ntx;
        c.org_z = c.org_y + g.nty;
        dim3 grid((unsigned)c.n_tiles, (unsigned)g.n_slabs);
#define CSL_VF_CASE(SV)                                                                        \
    case SV:                                                                                   \
        k_vf_grad<SV><<<grid, kVfThreads, 0, s>>>(L->rec.as<csl_rec>(),                        \
                                                  bins.vals.as<uint32_t>(),                    \
                                                  bins.tile_start.as<uint32_t>(),              \
                                                  bins.tile_end.as<uint32_t>(), c, grad_vf,    \
                                                  partial.as<float4>());                       \
        break;
        switch (cells.m) {
            CSL_VF_CASE(1)
            CSL_VF_CASE(2)
            CSL_VF_CASE(4)
            CSL_VF_CASE(8)
            default: fail(CSL_ERR_INVALID_ARG, "m must be 1, 2, 4 or 8");
        }
#undef CSL_VF_CASE
        CSL_LAUNCH_CHECK("vf gradient");
        // sum the partials per edge record in entry order
        DevBuf idx((size_t)bins.n_pairs * 4, s), tk((size_t)bins.n_pairs * 4, s),
            tv((size_t)bins.n_pairs * 4, s);
        k_iota<<<grid_for(bins.n_pairs, 256), 256, 0, s>>>(idx.as<uint32_t>(), bins.n_pairs);
        CSL_LAUNCH_CHECK("iota");
        radix_sort_pairs(bins.vals.as<uint32_t>(), idx.as<uint32_t>(), tk.as<uint32_t>(),
                         tv.as<uint32_t>(), bins.n_pairs, bits_for(ne), s);
        k_seg_sum<<<grid_for(bins.n_pairs, 256), 256, 0, s>>>(
            bins.vals.as<uint32_t>(), idx.as<uint32_t>(), bins.n_pairs, partial.as<float4>(),
            acc.as<float>());
        CSL_LAUNCH_CHECK("segment sums");
    }
    DevBuf gend((size_t)ne * 24, s);
    k_edge_out<<<grid_for(ne, 256), 256, 0, s>>>(
        acc.as<float>(), L->sid.as<uint32_t>(), L->radius.as<float>(), ne, L->R, L->C, L->mode,
        (float)(1.0 / (L->R * L->R * L->R * L->R)), grad_radius, gend.as<float>());
    CSL_LAUNCH_CHECK("edge gradients");
    if (!L->node_csr_off.get()) build_node_csr(L, s);
    k_node_grad<<<grid_for(nn, 256), 256, 0, s>>>(L->node_csr_off.as<int64_t>(),
                                                 L->node_csr.as<uint32_t>(), gend.as<float>(), nn,
                                                 grad_nodes);
    CSL_LAUNCH_CHECK("node gradients");
}

}  // namespace csl
