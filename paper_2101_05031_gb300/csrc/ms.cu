// Marching squares on each layer's Sigma image and assembly of closed loops
// (Sec. 4, last paragraph: the binary image is traced by marching squares).
//
// Grid: pixel samples padded by one ring of outside samples (padded sample
// (I, J) is pixel (I-1, J-1)), so every contour closes. Grid-edge ids are
// 2 (J W + I) (+1 for the vertical edge), W = nx + 2.
//   1. k_edge_bits: one bit per grid edge, set where the two samples differ
//      in inside-ness (Sigma >= C); 32 edges per word, a warp assembles two
//      words from two ballots.
//   2. a prefix sum of the words' popcounts gives every crossing a dense id,
//      in (layer, edge id) order: id(e) = prefix[word] + popc(lower bits).
//   3. k_emit: per cell, the vertices on the cell's own two edges (linear
//      interpolation of Sigma - C) and, for every side where a contour enters
//      the cell, its successor: walking the sides counter-clockwise, a side
//      from an inside to an outside corner is an entry, from outside to
//      inside an exit; a saddle (two inside corners on a diagonal) joins its
//      inside corners when the mean of the 4 corners is >= C, i.e. each entry
//      turns to the next side, else to the previous one. Inside is on the left.
//   4. k_heads: the head of a loop is its smallest dense id. Only local
//      minima (pred > id < succ) can be heads; each walks its loop until it
//      meets a smaller id (not the head) or returns (the head, which then
//      knows the loop length).
//   5. a prefix sum over (is_head, length) pairs gives each head its loop
//      index and first vertex; k_write walks each loop from its head and
//      writes the vertices contiguously.
#include <math.h>

#include "slice.cuh"

namespace csl {
namespace {

struct MsConst {
    int32_t nx, ny, W, H;
    int64_t words_per_layer;   // multiple of 2: 64 samples per warp
    int32_t n_layers;
    float C, fx0, fy0, fpx;
};

__device__ __forceinline__ bool inside_at(const float* __restrict__ sg, const MsConst& c, int I,
                                          int J) {
    if (I < 1 || J < 1 || I > c.nx || J > c.ny) return false;
    return sg[(int64_t)(J - 1) * c.nx + (I - 1)] >= c.C;
}
__device__ __forceinline__ float value_at(const float* __restrict__ sg, const MsConst& c, int I,
                                          int J) {
    if (I < 1 || J < 1 || I > c.nx || J > c.ny) return 0.0f;
    return sg[(int64_t)(J - 1) * c.nx + (I - 1)];
}

__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// grid: x = warps over the padded samples of a layer (32 samples, i.e. 64
// edges, per warp), y = layer.
__global__ void k_edge_bits(const float* __restrict__ sigma, MsConst c,
                            uint32_t* __restrict__ words) {
    const int layer = blockIdx.y;
    const float* sg = sigma + (int64_t)layer * c.nx * c.ny;
    const int64_t n_samples = (int64_t)c.W * c.H;
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = c.words_per_layer / 2;
    for (int64_t wg = warp_global; wg < n_warps;
         wg += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t q = wg * 32 + lane;
        bool hb = false, vb = false;
        if (q < n_samples) {
            int I = (int)(q % c.W), J = (int)(q / c.W);
            bool a = inside_at(sg, c, I, J);
            if (I + 1 < c.W) hb = a != inside_at(sg, c, I + 1, J);
            if (J + 1 < c.H) vb = a != inside_at(sg, c, I, J + 1);
        }
        uint32_t hm = __ballot_sync(0xffffffffu, hb), vm = __ballot_sync(0xffffffffu, vb);
        if (lane == 0) {
            uint2 out;
            out.x = spread16(hm) | (spread16(vm) << 1);
            out.y = spread16(hm >> 16) | (spread16(vm >> 16) << 1);
            reinterpret_cast<uint2*>(words + (int64_t)layer * c.words_per_layer)[wg] = out;
        }
    }
}

__global__ void k_popc(const uint32_t* __restrict__ words, int64_t n, uint32_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = __popc(words[i]);
}

struct Dense {
    const uint32_t* words;
    const uint32_t* prefix;
    int64_t wpl;
    __device__ __forceinline__ bool has(int layer, int64_t e) const {
        return (words[layer * wpl + (e >> 5)] >> (e & 31)) & 1u;
    }
    __device__ __forceinline__ uint32_t id(int layer, int64_t e) const {
        int64_t w = layer * wpl + (e >> 5);
        return prefix[w] + __popc(words[w] & ((1u << (e & 31)) - 1u));
    }
};

__global__ void k_emit(const float* __restrict__ sigma, MsConst c, Dense D,
                       float2* __restrict__ xy, int32_t* __restrict__ eid,
                       uint32_t* __restrict__ succ) {
    const int layer = blockIdx.y;
    const float* sg = sigma + (int64_t)layer * c.nx * c.ny;
    const int64_t n_cells = (int64_t)(c.nx + 1) * (c.ny + 1);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_cells;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(q % (c.nx + 1)), J = (int)(q / (c.nx + 1));
        const int64_t eb = 2 * ((int64_t)J * c.W + I);           // bottom side h(I, J)
        const int64_t el = eb + 1;                               // left side v(I, J)
        const int64_t er = 2 * ((int64_t)J * c.W + I + 1) + 1;   // right side v(I+1, J)
        const int64_t et = 2 * ((int64_t)(J + 1) * c.W + I);     // top side h(I, J+1)
        const bool hb = D.has(layer, eb), hl = D.has(layer, el);
        const bool hr = D.has(layer, er), ht = D.has(layer, et);
        if (!(hb | hl | hr | ht)) continue;
        const float v0 = value_at(sg, c, I, J), v1 = value_at(sg, c, I + 1, J);
        const float v2 = value_at(sg, c, I + 1, J + 1), v3 = value_at(sg, c, I, J + 1);
        const bool in0 = inside_at(sg, c, I, J), in1 = inside_at(sg, c, I + 1, J);
        const bool in2 = inside_at(sg, c, I + 1, J + 1), in3 = inside_at(sg, c, I, J + 1);
        // vertices on the cell's own edges
        if (hb) {
            uint32_t id = D.id(layer, eb);
            // inside sample first: t from it towards the other
            float sa = in0 ? v0 : v1, sb = in0 ? v1 : v0;
            float t = (sa - c.C) / (sa - sb);
            float xp = in0 ? ((float)I - 0.5f + t) : ((float)I + 0.5f - t);
            xy[id] = make_float2(c.fx0 + xp * c.fpx, c.fy0 + ((float)J - 0.5f) * c.fpx);
            eid[id] = (int32_t)eb;
        }
        if (hl) {
            uint32_t id = D.id(layer, el);
            float sa = in0 ? v0 : v3, sb = in0 ? v3 : v0;
            float t = (sa - c.C) / (sa - sb);
            float yp = in0 ? ((float)J - 0.5f + t) : ((float)J + 0.5f - t);
            xy[id] = make_float2(c.fx0 + ((float)I - 0.5f) * c.fpx, c.fy0 + yp * c.fpx);
            eid[id] = (int32_t)el;
        }
        // successors: sides counter-clockwise 0 bottom, 1 right, 2 top, 3 left
        const bool in[4] = {in0, in1, in2, in3};
        const int64_t side[4] = {eb, er, et, el};
        int n_enter = 0, enter0 = -1, enter1 = -1, leave0 = -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            bool a = in[k], b = in[(k + 1) & 3];
            if (a && !b) {
                if (n_enter == 0) enter0 = k; else enter1 = k;
                ++n_enter;
            }
            if (!a && b && leave0 < 0) leave0 = k;
        }
        if (n_enter == 1) {
            succ[D.id(layer, side[enter0])] = D.id(layer, side[leave0]);
        } else if (n_enter == 2) {
            const bool joined = 0.25f * (v0 + v1 + v2 + v3) >= c.C;
            const int k0 = enter0, k1 = enter1;
            const int t0 = joined ? ((k0 + 1) & 3) : ((k0 + 3) & 3);
            const int t1 = joined ? ((k1 + 1) & 3) : ((k1 + 3) & 3);
            succ[D.id(layer, side[k0])] = D.id(layer, side[t0]);
            succ[D.id(layer, side[k1])] = D.id(layer, side[t1]);
        }
    }
}

// Every crossing must have received exactly one successor; anything else is
// reported through *status and nothing is written out of range.
__global__ void k_pred(const uint32_t* __restrict__ succ, int64_t n, uint32_t* __restrict__ pred,
                       uint32_t* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t s = succ[i];
        if ((int64_t)s < n) pred[s] = (uint32_t)i;
        else atomicOr(status, ST_CAPACITY);
    }
}

__global__ void k_heads(const uint32_t* __restrict__ succ, const uint32_t* __restrict__ pred,
                        int64_t n, int64_t* __restrict__ packed, uint32_t* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q = (uint32_t)i;
        int64_t v = 0;
        if (pred[q] > q && succ[q] > q) {
            uint32_t j = succ[q];
            int64_t len = 1;
            bool head = true;
            while (j != q) {
                if (j < q) { head = false; break; }
                j = succ[j];
                if (++len > n) {   // a successor chain that never returns: corrupt input
                    atomicOr(status, ST_CAPACITY);
                    head = false;
                    break;
                }
            }
            if (head) v = ((int64_t)1 << 32) | len;
        }
        packed[i] = v;
    }
}

__global__ void k_write(const uint32_t* __restrict__ succ, const int64_t* __restrict__ packed,
                        const int64_t* __restrict__ scan, const float2* __restrict__ xy,
                        const int32_t* __restrict__ eid, int64_t n, int64_t* __restrict__ loop_off,
                        float2* __restrict__ oxy, int32_t* __restrict__ oeid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = packed[i];
        if (p == 0) continue;
        const int64_t len = p & 0xffffffffLL;
        const int64_t loop = scan[i] >> 32;
        const int64_t voff = scan[i] & 0xffffffffLL;
        loop_off[loop] = voff;
        uint32_t j = (uint32_t)i;
        for (int64_t r = 0; r < len; ++r) {
            oxy[voff + r] = xy[j];
            if (oeid) oeid[voff + r] = eid[j];
            j = succ[j];
        }
    }
}

// layer_loops[l] = loops whose head lies before the first crossing of layer l
__global__ void k_layer_loops(const uint32_t* __restrict__ prefix, int64_t wpl, int n_layers,
                              const int64_t* __restrict__ scan, int64_t n_cross, int64_t n_loops,
                              int64_t* __restrict__ layer_loops, int64_t* __restrict__ loop_off) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > n_layers) return;
    int64_t first = l < n_layers ? (int64_t)prefix[(int64_t)l * wpl] : n_cross;
    layer_loops[l] = first < n_cross ? (scan[first] >> 32) : n_loops;
    if (l == 0) loop_off[n_loops] = n_cross;
}

}  // namespace

void contours_chunk(const ChunkGeom& g, double C, const float* sigma, bool want_eid,
                    ChunkContours& out, cudaStream_t s) {
    MsConst c;
    c.nx = g.nx;
    c.ny = g.ny;
    c.W = g.nx + 2;
    c.H = g.ny + 2;
    const int64_t n_samples = (int64_t)c.W * c.H;
    c.words_per_layer = 2 * ceil_div(n_samples, 32);
    c.n_layers = g.n_layers;
    c.C = (float)C;
    c.fx0 = (float)g.x0;
    c.fy0 = (float)g.y0;
    c.fpx = (float)g.px;
    const int64_t n_words = c.words_per_layer * g.n_layers;
    if (n_words >= ((int64_t)1 << 27)) fail(CSL_ERR_CAPACITY, "marching squares: chunk too large");

    DevBuf words((size_t)n_words * 4, s), prefix((size_t)n_words * 4, s), total(8, s);
    {
        int64_t warps = c.words_per_layer / 2;
        dim3 grid(grid_for(warps * 32, 256, 2048), (unsigned)g.n_layers);
        k_edge_bits<<<grid, 256, 0, s>>>(sigma, c, words.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms edge bits");
    }
    k_popc<<<grid_for(n_words, 256), 256, 0, s>>>(words.as<uint32_t>(), n_words,
                                                  prefix.as<uint32_t>());
    CSL_LAUNCH_CHECK("ms popc");
    // 32-bit dense ids: n_words < 2^27 keeps every count below 2^32
    exclusive_scan_u32(prefix.as<uint32_t>(), prefix.as<uint32_t>(), n_words, total.as<uint32_t>(),
                       s);
    uint32_t n_cross_u = 0;
    read_to_host(&n_cross_u, total.get(), 4, s);
    const int64_t n_cross = n_cross_u;
    out.n_verts = n_cross;
    out.layer_loops.ensure((size_t)(g.n_layers + 1) * 8, s);
    if (n_cross == 0) {
        CSL_CUDA(cudaMemsetAsync(out.layer_loops.get(), 0, (size_t)(g.n_layers + 1) * 8, s));
        out.n_loops = 0;
        out.loop_off.ensure(8, s);
        CSL_CUDA(cudaMemsetAsync(out.loop_off.get(), 0, 8, s));
        return;
    }
    DevBuf xy((size_t)n_cross * 8, s), eid((size_t)n_cross * 4, s), succ((size_t)n_cross * 4, s);
    CSL_CUDA(cudaMemsetAsync(succ.get(), 0xff, (size_t)n_cross * 4, s));
    Dense D{words.as<uint32_t>(), prefix.as<uint32_t>(), c.words_per_layer};
    {
        int64_t n_cells = (int64_t)(c.nx + 1) * (c.ny + 1);
        dim3 grid(grid_for(n_cells, 256, 4096), (unsigned)g.n_layers);
        k_emit<<<grid, 256, 0, s>>>(sigma, c, D, xy.as<float2>(), eid.as<int32_t>(),
                                    succ.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms emit");
    }
    DevBuf pred((size_t)n_cross * 4, s), packed((size_t)n_cross * 8, s), scan((size_t)n_cross * 8, s);
    DevBuf status(4, s);
    CSL_CUDA(cudaMemsetAsync(status.get(), 0, 4, s));
    CSL_CUDA(cudaMemsetAsync(pred.get(), 0xff, (size_t)n_cross * 4, s));
    k_pred<<<grid_for(n_cross, 256), 256, 0, s>>>(succ.as<uint32_t>(), n_cross, pred.as<uint32_t>(),
                                                  status.as<uint32_t>());
    CSL_LAUNCH_CHECK("ms pred");
    {
        uint32_t st0 = 0;
        read_to_host(&st0, status.get(), 4, s);
        if (st0) fail(CSL_ERR_CUDA, "marching squares: a crossing has no successor");
    }
    k_heads<<<grid_for(n_cross, 256), 256, 0, s>>>(succ.as<uint32_t>(), pred.as<uint32_t>(), n_cross,
                                                   packed.as<int64_t>(), status.as<uint32_t>());
    CSL_LAUNCH_CHECK("ms heads");
    DevBuf tot(8, s);
    exclusive_scan_i64(packed.as<int64_t>(), scan.as<int64_t>(), n_cross, tot.as<int64_t>(), s);
    int64_t packed_total = read_i64(tot.as<int64_t>(), s);
    uint32_t st = 0;
    read_to_host(&st, status.get(), 4, s);
    if (st) fail(CSL_ERR_CUDA, "marching squares: inconsistent successor links");
    const int64_t n_loops = packed_total >> 32;
    if ((packed_total & 0xffffffffLL) != n_cross)
        fail(CSL_ERR_CUDA, "marching squares: loops do not cover every crossing");
    out.n_loops = n_loops;
    out.loop_off.ensure((size_t)(n_loops + 1) * 8, s);
    out.xy.ensure((size_t)n_cross * 8, s);
    if (want_eid) out.eid.ensure((size_t)n_cross * 4, s);
    k_write<<<grid_for(n_cross, 256), 256, 0, s>>>(
        succ.as<uint32_t>(), packed.as<int64_t>(), scan.as<int64_t>(), xy.as<float2>(),
        eid.as<int32_t>(), n_cross, out.loop_off.as<int64_t>(), out.xy.as<float2>(),
        want_eid ? out.eid.as<int32_t>() : nullptr);
    CSL_LAUNCH_CHECK("ms write");
    k_layer_loops<<<(unsigned)ceil_div(g.n_layers + 1, 128), 128, 0, s>>>(
        prefix.as<uint32_t>(), c.words_per_layer, g.n_layers, scan.as<int64_t>(), n_cross, n_loops,
        out.layer_loops.as<int64_t>(), out.loop_off.as<int64_t>());
    CSL_LAUNCH_CHECK("ms layer loops");
}

}  // namespace csl
