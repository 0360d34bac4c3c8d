// Zigzag infill of every layer's contours (Sec. 6: after the binary image and
// its boundary contours, a zigzag toolpath fills the interior).
//
// Scan lines y_m = y0 + m * spacing (m < n_lines; the same in every layer; y_m
// is y0 + m spacing in double, rounded once to float). An edge a -> b of a
// loop crosses line m when min(a_y, b_y) <= y_m < max(a_y, b_y) (half-open,
// decided in float), at x = a_x + t (b_x - a_x), t = (y_m - a_y) / (b_y - a_y).
// Along each line the crossings, sorted by x, alternate between entering and
// leaving the solid (the loops are closed and do not cross), so consecutive
// pairs are the inside segments. The toolpath of a layer visits the lines in
// increasing m, the segments of even lines from low to high x and those of odd
// lines in the opposite order, each odd-line segment from high to low x.
//
// Device pipeline: loop and layer of every vertex (flags + scans), crossings
// per edge (count, scan, emit (key = layer * n_lines + m, x)), a stable radix
// sort by x and then by key, pairs into segments, run bounds per key, and the
// zigzag permutation.
#include <math.h>
#include <string.h>

#include <functional>
#include <new>

#include "common.cuh"

namespace csl {
namespace {

// The scan lines' y, computed once in double and rounded to float.
__global__ void k_line_table(double y0, double sp, int n, float* __restrict__ ys) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) ys[m] = (float)(y0 + (double)m * sp);
}

// first m in [0, n] with ys[m] >= v (the table is non-decreasing): a float
// estimate, then exact comparisons against the table
__device__ __forceinline__ int first_line_at_or_above(const float* __restrict__ ys, float y0f,
                                                      float inv_sp, int n, float v) {
    const float e = ceilf((v - y0f) * inv_sp);
    int m = e < 0.0f ? 0 : (e > (float)n ? n : (int)e);
    while (m > 0 && ys[m - 1] >= v) --m;
    while (m < n && ys[m] < v) ++m;
    return m;
}

__global__ void k_mark_i64(const int64_t* __restrict__ off, int64_t n_groups, int64_t n_items,
                           uint32_t* __restrict__ flag) {
    // flag[off[g]] += 1 for every group g >= 1 that starts inside [0, n_items)
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; g < n_groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = off[g];
        if (p >= 0 && p < n_items) atomicAdd(flag + p, 1u);
    }
}

// inclusive scan from the exclusive one: idx[i] = excl[i] + flag[i]
__global__ void k_incl(const uint32_t* __restrict__ flag, uint32_t* __restrict__ idx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        idx[i] += flag[i];
}

struct HatchConst {
    const float* ys;   // the lines' y (k_line_table)
    float y0f, inv_sp;
    int32_t n_lines;
    int64_t n_verts;
};

__device__ __forceinline__ void edge_of(const int64_t* __restrict__ loop_off,
                                        const uint32_t* __restrict__ loop_of, int64_t v,
                                        int64_t& w) {
    const uint32_t L = loop_of[v];
    w = v + 1 < loop_off[L + 1] ? v + 1 : loop_off[L];
}

__global__ void k_count(const float2* __restrict__ xy, const int64_t* __restrict__ loop_off,
                        const uint32_t* __restrict__ loop_of, HatchConst c,
                        uint32_t* __restrict__ cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < c.n_verts;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t w;
        edge_of(loop_off, loop_of, v, w);
        const float ya = xy[v].y, yb = xy[w].y;
        const float lo = fminf(ya, yb), hi = fmaxf(ya, yb);
        uint32_t k = 0;
        if (lo < hi) {
            const int m0 = first_line_at_or_above(c.ys, c.y0f, c.inv_sp, c.n_lines, lo);
            const int m1 = first_line_at_or_above(c.ys, c.y0f, c.inv_sp, c.n_lines, hi);
            k = (uint32_t)(m1 - m0);
        }
        cnt[v] = k;
    }
}

__global__ void k_emit_crossings(const float2* __restrict__ xy, const int64_t* __restrict__ loop_off,
                                 const uint32_t* __restrict__ loop_of,
                                 const uint32_t* __restrict__ layer_of, HatchConst c,
                                 const int64_t* __restrict__ pos, uint32_t* __restrict__ key,
                                 float* __restrict__ xs) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < c.n_verts;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t w;
        edge_of(loop_off, loop_of, v, w);
        const float2 a = xy[v], b = xy[w];
        const float lo = fminf(a.y, b.y), hi = fmaxf(a.y, b.y);
        if (!(lo < hi)) continue;
        const int m0 = first_line_at_or_above(c.ys, c.y0f, c.inv_sp, c.n_lines, lo);
        const int m1 = first_line_at_or_above(c.ys, c.y0f, c.inv_sp, c.n_lines, hi);
        const uint32_t base = layer_of[loop_of[v]] * (uint32_t)c.n_lines;
        int64_t p = pos[v];
        for (int m = m0; m < m1; ++m, ++p) {
            const float ym = c.ys[m];
            const float t = __fdiv_rn(ym - a.y, b.y - a.y);
            key[p] = base + (uint32_t)m;
            xs[p] = fmaf(t, b.x - a.x, a.x);
        }
    }
}

// float -> uint32 whose unsigned order is the float order
__global__ void k_x_keys(const float* __restrict__ xs, int64_t n, uint32_t* __restrict__ k,
                         uint32_t* __restrict__ idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = __float_as_uint(xs[i]);
        k[i] = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_gather_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx,
                             int64_t n, uint32_t* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

// Segment s = sorted crossings (2s, 2s + 1), which must lie on one line.
__global__ void k_pairs(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sidx,
                        const float* __restrict__ xs, int64_t n_seg,
                        uint32_t* __restrict__ seg_key, float2* __restrict__ seg_x,
                        uint32_t* status) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k0 = skey[2 * s], k1 = skey[2 * s + 1];
        if (k0 != k1) atomicOr(status, ST_CAPACITY);   // a line with an odd crossing count
        seg_key[s] = k0;
        seg_x[s] = make_float2(xs[sidx[2 * s]], xs[sidx[2 * s + 1]]);
    }
}

__global__ void k_runs(const uint32_t* __restrict__ seg_key, int64_t n_seg,
                       uint32_t* __restrict__ run_lo, uint32_t* __restrict__ run_hi) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = seg_key[s];
        if (s == 0 || seg_key[s - 1] != k) run_lo[k] = (uint32_t)s;
        if (s == n_seg - 1 || seg_key[s + 1] != k) run_hi[k] = (uint32_t)(s + 1);
    }
}

__global__ void k_zigzag(const uint32_t* __restrict__ seg_key, const float2* __restrict__ seg_x,
                         const uint32_t* __restrict__ run_lo, const uint32_t* __restrict__ run_hi,
                         int64_t n_seg, HatchConst c, float* __restrict__ out) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = seg_key[s];
        const int m = (int)(k % (uint32_t)c.n_lines);
        const float2 x = seg_x[s];
        const bool odd = (m & 1) != 0;
        const int64_t o = odd ? (int64_t)run_lo[k] + run_hi[k] - 1 - s : s;
        out[3 * o] = odd ? x.y : x.x;
        out[3 * o + 1] = odd ? x.x : x.y;
        out[3 * o + 2] = c.ys[m];
    }
}

// layer_off[k] = first segment of layer k (keys k * n_lines ...)
__global__ void k_layer_offsets(const uint32_t* __restrict__ seg_key, int64_t n_seg, int n_layers,
                                int n_lines, int64_t* __restrict__ layer_off) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_layers) return;
    const uint32_t target = (uint32_t)k * (uint32_t)n_lines;
    int64_t lo = 0, hi = n_seg;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (seg_key[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    layer_off[k] = k == n_layers ? n_seg : lo;
}

int bits_for(uint64_t n) {
    int b = 1;
    while (b < 32 && ((uint64_t)1 << b) < n) ++b;
    return b;
}

}  // namespace
}  // namespace csl

using namespace csl;

extern "C" {

csl_status csl_hatch_layers(const csl_contours* ct, double y0, double spacing, int32_t n_lines,
                            int32_t dst_on_device, void* stream, csl_hatches** out) {
    try {
        if (!out) fail(CSL_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (!ct) fail(CSL_ERR_INVALID_ARG, "contours is NULL");
        if (!ct->on_device) fail(CSL_ERR_INVALID_ARG, "contours must be on the device");
        if (!(isfinite(y0) && isfinite(spacing) && spacing > 0.0))
            fail(CSL_ERR_INVALID_ARG, "y0 must be finite and spacing > 0");
        if (n_lines < 0) fail(CSL_ERR_INVALID_ARG, "n_lines < 0");
        const int64_t n_layers = ct->n_layers, n_loops = ct->n_loops, n_verts = ct->n_verts;
        if ((uint64_t)n_layers * (uint64_t)(n_lines > 0 ? n_lines : 1) >= 0xffffffffull)
            fail(CSL_ERR_CAPACITY, "n_layers * n_lines must be below 2^32");
        if (n_verts >= 0xffffffffLL || n_loops >= 0xffffffffLL)
            fail(CSL_ERR_CAPACITY, "too many vertices");
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf ys_d((size_t)(n_lines > 0 ? n_lines : 1) * 4, s);
        if (n_lines > 0) {
            k_line_table<<<(unsigned)ceil_div(n_lines, 256), 256, 0, s>>>(y0, spacing, n_lines,
                                                                         ys_d.as<float>());
            CSL_LAUNCH_CHECK("hatch lines");
        }
        HatchConst c{ys_d.as<float>(), (float)y0, (float)(1.0 / spacing), n_lines, n_verts};
        const float2* xy = reinterpret_cast<const float2*>(ct->xy);

        int64_t n_rec = 0;
        DevBuf key, xs, small(16, s);
        CSL_CUDA(cudaMemsetAsync(small.get(), 0, 16, s));
        if (n_verts > 0 && n_lines > 0) {
            // loop of every vertex, layer of every loop
            DevBuf vflag((size_t)n_verts * 4, s), loop_of((size_t)n_verts * 4, s);
            CSL_CUDA(cudaMemsetAsync(vflag.get(), 0, (size_t)n_verts * 4, s));
            k_mark_i64<<<grid_for(n_loops, 256), 256, 0, s>>>(ct->loop_vert_off, n_loops, n_verts,
                                                              vflag.as<uint32_t>());
            CSL_LAUNCH_CHECK("hatch loop starts");
            exclusive_scan_u32(vflag.as<uint32_t>(), loop_of.as<uint32_t>(), n_verts, nullptr, s);
            k_incl<<<grid_for(n_verts, 256), 256, 0, s>>>(vflag.as<uint32_t>(),
                                                          loop_of.as<uint32_t>(), n_verts);
            CSL_LAUNCH_CHECK("hatch loop of vertex");
            DevBuf lflag((size_t)n_loops * 4, s), layer_of((size_t)n_loops * 4, s);
            CSL_CUDA(cudaMemsetAsync(lflag.get(), 0, (size_t)n_loops * 4, s));
            k_mark_i64<<<grid_for(n_layers, 256), 256, 0, s>>>(ct->layer_loop_off, n_layers,
                                                               n_loops, lflag.as<uint32_t>());
            CSL_LAUNCH_CHECK("hatch layer starts");
            exclusive_scan_u32(lflag.as<uint32_t>(), layer_of.as<uint32_t>(), n_loops, nullptr, s);
            k_incl<<<grid_for(n_loops, 256), 256, 0, s>>>(lflag.as<uint32_t>(),
                                                          layer_of.as<uint32_t>(), n_loops);
            CSL_LAUNCH_CHECK("hatch layer of loop");
            // the first loops may precede the first layer start only when layer 0
            // has loops; layer_loop_off[0] is 0, so the counts are the layers
            DevBuf cnt((size_t)n_verts * 4, s), pos((size_t)n_verts * 8, s);
            k_count<<<grid_for(n_verts, 256), 256, 0, s>>>(xy, ct->loop_vert_off,
                                                           loop_of.as<uint32_t>(), c,
                                                           cnt.as<uint32_t>());
            CSL_LAUNCH_CHECK("hatch count");
            exclusive_scan_u32_to_i64(cnt.as<uint32_t>(), pos.as<int64_t>(), n_verts,
                                      small.as<int64_t>(), s);
            n_rec = read_i64(small.as<int64_t>(), s);
            if (n_rec >= 0xffffffffLL) fail(CSL_ERR_CAPACITY, "too many crossings");
            if (n_rec % 2) fail(CSL_ERR_CUDA, "hatching: odd number of crossings");
            key.alloc((size_t)(n_rec ? n_rec : 1) * 4, s);
            xs.alloc((size_t)(n_rec ? n_rec : 1) * 4, s);
            if (n_rec)
                k_emit_crossings<<<grid_for(n_verts, 256), 256, 0, s>>>(
                    xy, ct->loop_vert_off, loop_of.as<uint32_t>(), layer_of.as<uint32_t>(), c,
                    pos.as<int64_t>(), key.as<uint32_t>(), xs.as<float>());
            CSL_LAUNCH_CHECK("hatch crossings");
        }
        const int64_t n_seg = n_rec / 2;
        const uint64_t n_keys = (uint64_t)n_layers * (uint64_t)(n_lines > 0 ? n_lines : 1);

        csl_hatches* h = new csl_hatches();
        memset(h, 0, sizeof(*h));
        h->n_layers = (int32_t)n_layers;
        h->on_device = dst_on_device ? 1 : 0;
        h->n_segments = n_seg;
        auto alloc = [&](void** p, size_t b) {
            if (dst_on_device) {
                if (cudaMalloc(p, b ? b : 16) != cudaSuccess) {
                    cudaGetLastError();
                    fail(CSL_ERR_OOM, "device allocation of the hatches failed");
                }
            } else {
                *p = host_block_alloc(b ? b : 16);
            }
        };
        try {
            alloc((void**)&h->layer_seg_off, (size_t)(n_layers + 1) * 8);
            alloc((void**)&h->seg, (size_t)n_seg * 12);
            DevBuf lay((size_t)(n_layers + 1) * 8, s), segs((size_t)(n_seg ? n_seg : 1) * 12, s);
            if (n_seg > 0) {
                // sort by x, then (stably) by line key
                DevBuf k1((size_t)n_rec * 4, s), idx((size_t)n_rec * 4, s), tk((size_t)n_rec * 4, s),
                    tv((size_t)n_rec * 4, s);
                k_x_keys<<<grid_for(n_rec, 256), 256, 0, s>>>(xs.as<float>(), n_rec,
                                                              k1.as<uint32_t>(), idx.as<uint32_t>());
                CSL_LAUNCH_CHECK("hatch x keys");
                radix_sort_pairs(k1.as<uint32_t>(), idx.as<uint32_t>(), tk.as<uint32_t>(),
                                 tv.as<uint32_t>(), n_rec, 32, s);
                k_gather_u32<<<grid_for(n_rec, 256), 256, 0, s>>>(key.as<uint32_t>(),
                                                                  idx.as<uint32_t>(), n_rec,
                                                                  k1.as<uint32_t>());
                CSL_LAUNCH_CHECK("hatch gather keys");
                radix_sort_pairs(k1.as<uint32_t>(), idx.as<uint32_t>(), tk.as<uint32_t>(),
                                 tv.as<uint32_t>(), n_rec, bits_for(n_keys), s);
                DevBuf seg_key((size_t)n_seg * 4, s), seg_x((size_t)n_seg * 8, s);
                k_pairs<<<grid_for(n_seg, 256), 256, 0, s>>>(k1.as<uint32_t>(), idx.as<uint32_t>(),
                                                             xs.as<float>(), n_seg,
                                                             seg_key.as<uint32_t>(),
                                                             seg_x.as<float2>(),
                                                             small.as<uint32_t>() + 2);
                CSL_LAUNCH_CHECK("hatch pairs");
                DevBuf run_lo((size_t)n_keys * 4, s), run_hi((size_t)n_keys * 4, s);
                k_runs<<<grid_for(n_seg, 256), 256, 0, s>>>(seg_key.as<uint32_t>(), n_seg,
                                                            run_lo.as<uint32_t>(),
                                                            run_hi.as<uint32_t>());
                CSL_LAUNCH_CHECK("hatch runs");
                k_zigzag<<<grid_for(n_seg, 256), 256, 0, s>>>(seg_key.as<uint32_t>(),
                                                              seg_x.as<float2>(),
                                                              run_lo.as<uint32_t>(),
                                                              run_hi.as<uint32_t>(), n_seg, c,
                                                              segs.as<float>());
                CSL_LAUNCH_CHECK("hatch zigzag");
                k_layer_offsets<<<(unsigned)ceil_div(n_layers + 1, 128), 128, 0, s>>>(
                    seg_key.as<uint32_t>(), n_seg, (int)n_layers, n_lines, lay.as<int64_t>());
                CSL_LAUNCH_CHECK("hatch layer offsets");
                uint32_t st = 0;
                read_to_host(&st, small.as<uint32_t>() + 2, 4, s);
                if (st) fail(CSL_ERR_CUDA, "hatching: a line with an odd number of crossings");
            } else {
                CSL_CUDA(cudaMemsetAsync(lay.get(), 0, (size_t)(n_layers + 1) * 8, s));
            }
            const cudaMemcpyKind kind =
                dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            CSL_CUDA(cudaMemcpyAsync(h->layer_seg_off, lay.get(), (size_t)(n_layers + 1) * 8,
                                     kind, s));
            if (n_seg)
                CSL_CUDA(cudaMemcpyAsync(h->seg, segs.get(), (size_t)n_seg * 12, kind, s));
            CSL_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            csl_hatches_free(h);
            throw;
        }
        *out = h;
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

void csl_hatches_free(csl_hatches* h) {
    if (!h) return;
    if (h->on_device) {
        cudaFree(h->layer_seg_off);
        cudaFree(h->seg);
    } else {
        host_block_free(h->layer_seg_off);
        host_block_free(h->seg);
    }
    delete h;
}

}  // extern "C"
