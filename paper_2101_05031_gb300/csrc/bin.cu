// Slab / tile binner. The active-edge set of Eq. 8 is widened from one plane
// to a slab of S layers, then split over 2D tiles of 16 x 16 pixels:
//   1. per slab, a window of the v_s^z-sorted records (binary search);
//   2. per (slab, record): the FP32 bin predicate below -> a rectangle of tiles,
//      counted, prefix-summed and emitted as (slab * n_tiles + tile, record);
//   3. a stable radix sort by that key, so every (slab, tile) list is
//      contiguous and in record order (deterministic);
//   4. list boundaries per key.
//
// Bin predicate (all FP32, round-to-nearest, no fused operations), for a slab
// whose first and last layer planes are zf <= zl and an edge with exact
// endpoints (ax, ay, zlo) -> (bx, by, zhi), zlo <= zhi:
//   reject unless (zlo - mz) <= zl and (zhi + mz) >= zf;
//   t0 = 0, t1 = 1; if zhi - zlo > 0:
//       t0 = max(((zf - mz) - zlo) / (zhi - zlo), 0), t1 = min(((zl + mz) - zlo) / (zhi - zlo), 1)
//   x(t) = ax + t (bx - ax), y(t) likewise;
//   box = [min(x(t0), x(t1)) - mxy, max(...) + mxy] x [same in y];
//   tile range = floor((box - origin) * inv_tile), clipped to the grid; with a
//   one-pixel halo (the fused field and contour pass, which also evaluates each
//   tile's next column and row) the low corner is floor(((min - mxy) - px -
//   origin) * inv_tile).
// mz and mxy are R plus a slack for FP32 rounding, so every pixel centre of
// the tile (and of its halo) within distance R of the edge at some layer of
// the slab is inside.
#include <math.h>

#include "slice.cuh"

namespace csl {
namespace {

struct BinConst {
    float fx0, fy0, inv_tile, mxy, mz;
    float halo;   // 0, or the pixel size: the low corner also reaches the tile below
    int32_t ntx, nty, n_tiles;
    int32_t tb;   // > 0: entries carry slab << tb | tile and are sorted by the tile bits
};

struct SlabInfo {
    int64_t kb, ke;      // record window
    int64_t cand_off;    // first candidate of this slab
    float zf, zl;        // first / last layer plane of the slab
};

__device__ __forceinline__ bool bin_rect(const float4 e, float zlo, float zhi, float zf, float zl,
                                         const BinConst& c, int& tx0, int& tx1, int& ty0,
                                         int& ty1) {
    if (__fsub_rn(zlo, c.mz) > zl) return false;
    if (__fadd_rn(zhi, c.mz) < zf) return false;
    float t0 = 0.0f, t1 = 1.0f;
    float dzs = __fsub_rn(zhi, zlo);
    if (dzs > 0.0f) {
        t0 = fmaxf(__fdiv_rn(__fsub_rn(__fsub_rn(zf, c.mz), zlo), dzs), 0.0f);
        t1 = fminf(__fdiv_rn(__fsub_rn(__fadd_rn(zl, c.mz), zlo), dzs), 1.0f);
    }
    float ex = __fsub_rn(e.z, e.x), ey = __fsub_rn(e.w, e.y);
    float xa = __fadd_rn(e.x, __fmul_rn(t0, ex)), xb = __fadd_rn(e.x, __fmul_rn(t1, ex));
    float ya = __fadd_rn(e.y, __fmul_rn(t0, ey)), yb = __fadd_rn(e.y, __fmul_rn(t1, ey));
    float xmin = __fsub_rn(fminf(xa, xb), c.mxy), xmax = __fadd_rn(fmaxf(xa, xb), c.mxy);
    float ymin = __fsub_rn(fminf(ya, yb), c.mxy), ymax = __fadd_rn(fmaxf(ya, yb), c.mxy);
    if (c.halo > 0.0f) {
        xmin = __fsub_rn(xmin, c.halo);
        ymin = __fsub_rn(ymin, c.halo);
    }
    float fx0 = floorf(__fmul_rn(__fsub_rn(xmin, c.fx0), c.inv_tile));
    float fx1 = floorf(__fmul_rn(__fsub_rn(xmax, c.fx0), c.inv_tile));
    float fy0 = floorf(__fmul_rn(__fsub_rn(ymin, c.fy0), c.inv_tile));
    float fy1 = floorf(__fmul_rn(__fsub_rn(ymax, c.fy0), c.inv_tile));
    if (fx1 < 0.0f || fy1 < 0.0f || fx0 >= (float)c.ntx || fy0 >= (float)c.nty) return false;
    tx0 = (int)fmaxf(fx0, 0.0f);
    ty0 = (int)fmaxf(fy0, 0.0f);
    tx1 = (int)fminf(fx1, (float)(c.ntx - 1));
    ty1 = (int)fminf(fy1, (float)(c.nty - 1));
    return true;
}

// First / last layer plane of each slab, from double (non-fused, as the
// binning reference computes them) rounded to float.
__global__ void k_init_slabs(SlabInfo* slabs, int n_slabs, double z0, double dz, int first_layer,
                             int S, int last_layer) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= n_slabs) return;
    const int l0 = first_layer + sl * S;
    const int l1 = min(l0 + S - 1, last_layer);
    slabs[sl].zf = (float)__dadd_rn(z0, __dmul_rn((double)l0, dz));
    slabs[sl].zl = (float)__dadd_rn(z0, __dmul_rn((double)l1, dz));
    slabs[sl].kb = slabs[sl].ke = slabs[sl].cand_off = 0;
}

// Window of records for each slab: zlo in [zf - mz - max_dz - slack, zl + mz + slack].
__global__ void k_slab_windows(const float* __restrict__ zlo, int64_t n, SlabInfo* slabs,
                               int n_slabs, float mz, float max_dz) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slabs) return;
    float zf = slabs[s].zf, zl = slabs[s].zl;
    double lo_key = (double)zf - mz - max_dz - 1e-3 * (1.0 + fabs((double)zf));
    double hi_key = (double)zl + mz + 1e-3 * (1.0 + fabs((double)zl));
    int64_t a = 0, b = n;   // first k with zlo[k] >= lo_key
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if ((double)zlo[m] < lo_key) a = m + 1; else b = m;
    }
    int64_t kb = a;
    a = kb;
    b = n;                  // first k with zlo[k] > hi_key
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if ((double)zlo[m] <= hi_key) a = m + 1; else b = m;
    }
    slabs[s].kb = kb;
    slabs[s].ke = a;
}

__global__ void k_cand_offsets(SlabInfo* slabs, int n_slabs, int64_t* total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int s = 0; s < n_slabs; ++s) {
        slabs[s].cand_off = acc;
        acc += slabs[s].ke - slabs[s].kb;
    }
    *total = acc;
}

__global__ void k_bin_count(const float4* __restrict__ bxy, const float* __restrict__ zlo,
                            const float* __restrict__ zhi, const SlabInfo* __restrict__ slabs,
                            BinConst c, uint32_t* __restrict__ count, int64_t cap_cand,
                            uint32_t* flag) {
    const SlabInfo sl = slabs[blockIdx.y];
    int64_t n = sl.ke - sl.kb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = sl.kb + i;
        int tx0, tx1, ty0, ty1;
        uint32_t cnt = 0;
        if (bin_rect(bxy[k], zlo[k], zhi[k], sl.zf, sl.zl, c, tx0, tx1, ty0, ty1))
            cnt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        if (sl.cand_off + i < cap_cand) count[sl.cand_off + i] = cnt;
        else if (flag) atomicOr(flag, 1u);
    }
}

// Replay check: the device's totals must equal the planned ones.
__global__ void k_check_i64(const int64_t* __restrict__ v, int64_t expect, uint32_t* flag) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *v != expect) atomicOr(flag, 1u);
}

__global__ void k_check_windows(const SlabInfo* __restrict__ slabs, int n_slabs,
                                int64_t max_window, uint32_t* flag) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl < n_slabs && slabs[sl].ke - slabs[sl].kb > max_window) atomicOr(flag, 1u);
}

__global__ void k_bin_emit(const float4* __restrict__ bxy, const float* __restrict__ zlo,
                           const float* __restrict__ zhi, const SlabInfo* __restrict__ slabs,
                           BinConst c, const int64_t* __restrict__ pair_off, int64_t cap_cand,
                           int64_t cap_pairs, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
    const int s = blockIdx.y;
    const SlabInfo sl = slabs[s];
    int64_t n = sl.ke - sl.kb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = sl.kb + i;
        int tx0, tx1, ty0, ty1;
        if (!bin_rect(bxy[k], zlo[k], zhi[k], sl.zf, sl.zl, c, tx0, tx1, ty0, ty1)) continue;
        if (sl.cand_off + i >= cap_cand) continue;   // a replay whose sizes changed (flagged)
        int64_t p = pair_off[sl.cand_off + i];
        if (p + (int64_t)(tx1 - tx0 + 1) * (ty1 - ty0 + 1) > cap_pairs) continue;
        const uint32_t kbase = c.tb ? (uint32_t)s << c.tb : (uint32_t)s * (uint32_t)c.n_tiles;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                keys[p] = kbase + (uint32_t)(ty * c.ntx + tx);
                vals[p] = (uint32_t)k;
                ++p;
            }
    }
}

// [start, end) of every (slab, tile) run, at the bin index slab * n_tiles +
// tile (keys in either form of BinConst::tb).
__global__ void k_list_bounds(const uint32_t* __restrict__ keys, int64_t n, int tb, int n_tiles,
                              uint32_t* __restrict__ start, uint32_t* __restrict__ end) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        const uint32_t b =
            tb ? (k >> tb) * (uint32_t)n_tiles + (k & ((1u << tb) - 1u)) : k;
        if (i == 0 || keys[i - 1] != k) start[b] = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) end[b] = (uint32_t)(i + 1);
    }
}

// recs[p] = rec[vals[p]] (32 bytes each; an index out of range copies record 0)
__global__ void k_gather_records(const uint4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                 int64_t n, int64_t n_rec, uint4* __restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = vals[p];
        if ((int64_t)v >= n_rec) v = 0;   // only in a replay whose sizes changed (flagged)
        out[2 * p] = rec[2 * (int64_t)v];
        out[2 * p + 1] = rec[2 * (int64_t)v + 1];
    }
}

int bits_for(int64_t n) {
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) < n) ++b;
    return b;
}

}  // namespace

void bin_chunk(const csl_lattice* L, const ChunkGeom& g, SlabBins& out, cudaStream_t s,
               const Replay* rp) {
    const bool replay = rp && rp->replay;
    uint32_t* flag = rp ? rp->flag : nullptr;
    const int n_tiles = g.ntx * g.nty;
    const int64_t n_keys = (int64_t)g.n_slabs * n_tiles;
    if (n_keys > 0xffffffffLL) fail(CSL_ERR_CAPACITY, "too many (slab, tile) bins in one chunk");
    BinConst c;
    c.fx0 = (float)g.x0;
    c.fy0 = (float)g.y0;
    c.inv_tile = (float)(1.0 / ((double)g.T * g.px));
    c.mxy = g.margin_xy;
    c.mz = g.margin_z;
    c.halo = g.fused ? (float)g.px : 0.0f;
    c.ntx = g.ntx;
    c.nty = g.nty;
    c.n_tiles = n_tiles;
    // The entries are emitted slab by slab, so a stable sort by the tile alone
    // leaves every (slab, tile) run contiguous (tiles in order, slabs in order
    // within a tile) with its records in emission order: the same lists as a
    // sort by (slab, tile), in fewer passes. Keys then carry slab << tb | tile.
    const int tb = bits_for(n_tiles);
    c.tb = ((int64_t)g.n_slabs << tb) <= 0xffffffffLL && tb < bits_for(n_keys) ? std::max(tb, 1)
                                                                              : 0;

    std::vector<SlabInfo> hs(g.n_slabs);
    DevBuf slabs(sizeof(SlabInfo) * g.n_slabs, s);
    DevBuf total(sizeof(int64_t), s);
    k_init_slabs<<<(unsigned)ceil_div(g.n_slabs, 128), 128, 0, s>>>(
        slabs.as<SlabInfo>(), g.n_slabs, g.z0, g.dz, g.first_layer, g.S,
        g.first_layer + g.n_layers - 1);
    CSL_LAUNCH_CHECK("slab planes");
    k_slab_windows<<<(unsigned)ceil_div(g.n_slabs, 128), 128, 0, s>>>(
        L->zlo.as<float>(), L->n_edges, slabs.as<SlabInfo>(), g.n_slabs, c.mz, L->max_dz);
    CSL_LAUNCH_CHECK("slab windows");
    k_cand_offsets<<<1, 32, 0, s>>>(slabs.as<SlabInfo>(), g.n_slabs, total.as<int64_t>());
    CSL_LAUNCH_CHECK("candidate offsets");
    int64_t n_cand, max_window = 0;
    if (replay) {
        n_cand = rp->plan->n_cand;
        max_window = rp->plan->max_window;
        k_check_i64<<<1, 32, 0, s>>>(total.as<int64_t>(), n_cand, flag);
        CSL_LAUNCH_CHECK("check candidates");
        k_check_windows<<<(unsigned)ceil_div(g.n_slabs, 128), 128, 0, s>>>(
            slabs.as<SlabInfo>(), g.n_slabs, max_window, flag);
        CSL_LAUNCH_CHECK("check windows");
    } else {
        n_cand = read_i64(total.as<int64_t>(), s);
        read_to_host(hs.data(), slabs.get(), sizeof(SlabInfo) * g.n_slabs, s);
        for (auto& x : hs) max_window = std::max<int64_t>(max_window, x.ke - x.kb);
        if (rp) {
            rp->plan->n_cand = n_cand;
            rp->plan->max_window = max_window;
        }
    }

    out.n_cand = n_cand;
    out.tile_start.ensure((size_t)n_keys * 4, s);
    out.tile_end.ensure((size_t)n_keys * 4, s);
    CSL_CUDA(cudaMemsetAsync(out.tile_start.get(), 0, (size_t)n_keys * 4, s));
    CSL_CUDA(cudaMemsetAsync(out.tile_end.get(), 0, (size_t)n_keys * 4, s));
    out.n_pairs = 0;
    if (n_cand == 0) return;

    DevBuf count((size_t)n_cand * 4, s), pair_off((size_t)n_cand * 8, s);
    dim3 grid(grid_for(max_window, 256, 4096), (unsigned)g.n_slabs);
    k_bin_count<<<grid, 256, 0, s>>>(L->bxy.as<float4>(), L->zlo.as<float>(), L->zhi.as<float>(),
                                     slabs.as<SlabInfo>(), c, count.as<uint32_t>(), n_cand, flag);
    CSL_LAUNCH_CHECK("bin count");
    exclusive_scan_u32_to_i64(count.as<uint32_t>(), pair_off.as<int64_t>(), n_cand,
                              total.as<int64_t>(), s);
    int64_t n_pairs;
    if (replay) {
        n_pairs = rp->plan->n_pairs;
        k_check_i64<<<1, 32, 0, s>>>(total.as<int64_t>(), n_pairs, flag);
        CSL_LAUNCH_CHECK("check bin entries");
    } else {
        n_pairs = read_i64(total.as<int64_t>(), s);
        if (rp) rp->plan->n_pairs = n_pairs;
    }
    if (n_pairs > 0xffffffffLL) fail(CSL_ERR_CAPACITY, "more than 2^32 bin entries in one chunk");
    out.n_pairs = n_pairs;
    if (n_pairs == 0) return;
    out.keys.ensure((size_t)n_pairs * 4, s);
    out.vals.ensure((size_t)n_pairs * 4, s);
    k_bin_emit<<<grid, 256, 0, s>>>(L->bxy.as<float4>(), L->zlo.as<float>(), L->zhi.as<float>(),
                                    slabs.as<SlabInfo>(), c, pair_off.as<int64_t>(), n_cand,
                                    n_pairs, out.keys.as<uint32_t>(), out.vals.as<uint32_t>());
    CSL_LAUNCH_CHECK("bin emit");
    count.release();
    pair_off.release();
    {
        DevBuf tk((size_t)n_pairs * 4, s), tv((size_t)n_pairs * 4, s);
        radix_sort_pairs(out.keys.as<uint32_t>(), out.vals.as<uint32_t>(), tk.as<uint32_t>(),
                         tv.as<uint32_t>(), n_pairs, c.tb ? c.tb : bits_for(n_keys), s);
    }
    k_list_bounds<<<grid_for(n_pairs, 256), 256, 0, s>>>(out.keys.as<uint32_t>(), n_pairs, c.tb,
                                                        n_tiles, out.tile_start.as<uint32_t>(),
                                                        out.tile_end.as<uint32_t>());
    CSL_LAUNCH_CHECK("list bounds");
    // the records themselves in entry order, so that the field kernel stages a
    // tile's list with one bulk copy
    out.recs.ensure((size_t)n_pairs * sizeof(csl_rec), s);
    k_gather_records<<<grid_for(n_pairs, 256), 256, 0, s>>>(
        reinterpret_cast<const uint4*>(L->rec.get()), out.vals.as<uint32_t>(), n_pairs,
        L->n_edges, reinterpret_cast<uint4*>(out.recs.get()));
    CSL_LAUNCH_CHECK("gather records");
}

}  // namespace csl
