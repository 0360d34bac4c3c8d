// Marching squares on each layer's binary image and assembly of closed loops
// (Sec. 4, last paragraph: the binary image is traced by marching squares).
//
// Grid: pixel samples padded by one ring of outside samples (padded sample
// (I, J) is pixel (I-1, J-1)), so every contour closes. Grid-edge ids are
// 2 (J W + I) for the edge to (I+1, J) and 2 (J W + I) + 1 for the edge to
// (I, J+1), W = nx + 2. The field kernel leaves the inside mask (one bit per
// padded sample, rows of 32-bit words).
//   1. k_edge_words: per mask word (32 samples of one row), the crossing bits
//      of their two grid edges by shift and xor, interleaved (h, v) into two
//      32-bit edge words per mask word;
//   2. a prefix sum of the edge words' popcounts numbers the crossings in
//      (layer, edge id) order: id = prefix[word] + popc(lower bits);
//   3. k_emit: per mask word, only the cells with a crossing side: the vertex
//      on each of the cell's own two edges (the zero of the linear interpolant
//      of Sigma - C) and, for each side where a contour enters the cell, its
//      successor. Walking the sides counter-clockwise, a side from an inside
//      to an outside corner is an entry, from outside to inside an exit; a
//      saddle (two inside corners on a diagonal) joins its inside corners when
//      the mean of the 4 corner values is >= C, i.e. each entry turns to the
//      next side, else to the previous one. Inside lies on the left.
//   4. the head of a loop is its smallest id. Only local minima
//      (pred > id < succ) can be heads; they are compacted into a list and
//      each walks its loop until it meets a smaller id (not the head) or
//      returns (the head, which then knows the loop length);
//   5. a prefix sum over (is head, length) gives each head its loop index and
//      first vertex; each head walks its loop again and writes its vertices.
// Crossings are 16-byte records {x, y, successor, edge id}, so one walk step
// is one load.
#include <math.h>

#include <algorithm>

#include "slice.cuh"

namespace csl {
namespace {

struct MsConst {
    int32_t nx, ny, W, H;
    int32_t mwr;          // mask words per row
    int32_t ewr;          // edge words per row (2 per mask word)
    int64_t mask_wpl;     // mask words per layer
    int64_t edge_wpl;     // edge words per layer
    int32_t n_layers;
    float C, fx0, fy0, fpx;
};

struct __align__(16) Xing {
    float x, y;
    uint32_t succ;
    int32_t eid;
};

__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// grid: x over (row J, mask word k), y = layer
__global__ void k_edge_words(const uint32_t* __restrict__ mask, MsConst c,
                             uint32_t* __restrict__ ew) {
    const int layer = blockIdx.y;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint32_t)c.H * (uint32_t)c.mwr) return;
    const int J = (int)(idx / (uint32_t)c.mwr), k = (int)(idx - (uint32_t)J * c.mwr);
    const uint32_t* m = mask + (int64_t)layer * c.mask_wpl;
    const uint32_t in0 = m[(int64_t)J * c.mwr + k];
    const uint32_t in1 = k + 1 < c.mwr ? m[(int64_t)J * c.mwr + k + 1] : 0u;
    const uint32_t up = J + 1 < c.H ? m[(int64_t)(J + 1) * c.mwr + k] : 0u;
    const uint32_t h = in0 ^ ((in0 >> 1) | (in1 << 31));   // edge to (I+1, J)
    const uint32_t v = in0 ^ up;                           // edge to (I, J+1)
    uint2 out;
    out.x = spread16(h) | (spread16(v) << 1);
    out.y = spread16(h >> 16) | (spread16(v >> 16) << 1);
    reinterpret_cast<uint2*>(ew + (int64_t)layer * c.edge_wpl + (int64_t)J * c.ewr)[k] = out;
}

__global__ void k_popc(const uint32_t* __restrict__ words, int64_t n, uint32_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = __popc(words[i]);
}

struct Dense {
    const uint32_t* ew;
    const uint32_t* prefix;
    int64_t edge_wpl;
    int32_t ewr;
    // id of the crossing on edge (I, J, b), b = 0 horizontal, 1 vertical
    __device__ __forceinline__ uint32_t id(int layer, int I, int J, int b) const {
        const int64_t w = layer * edge_wpl + (int64_t)J * ewr + (I >> 4);
        const int bit = 2 * (I & 15) + b;
        return prefix[w] + __popc(ew[w] & ((1u << bit) - 1u));
    }
};

__device__ __forceinline__ float value_at(const float* __restrict__ sg, const MsConst& c, int I,
                                          int J) {
    if (I < 1 || J < 1 || I > c.nx || J > c.ny) return 0.0f;
    return sg[(int64_t)(J - 1) * c.nx + (I - 1)];
}

// grid: x over (row J <= ny, mask word k), y = layer
__global__ void k_emit(const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
                       MsConst c, Dense D, Xing* __restrict__ rec) {
    const int layer = blockIdx.y;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint32_t)(c.ny + 1) * (uint32_t)c.mwr) return;
    const int J = (int)(idx / (uint32_t)c.mwr), k = (int)(idx - (uint32_t)J * c.mwr);
    const uint32_t* m = mask + (int64_t)layer * c.mask_wpl;
    const float* sg = sigma + (int64_t)layer * c.nx * c.ny;
    const bool last = k + 1 >= c.mwr;
    const uint32_t in0 = m[(int64_t)J * c.mwr + k];
    const uint32_t in1 = last ? 0u : m[(int64_t)J * c.mwr + k + 1];
    const uint32_t up = m[(int64_t)(J + 1) * c.mwr + k];          // J + 1 <= ny + 1 < H
    const uint32_t up1 = last ? 0u : m[(int64_t)(J + 1) * c.mwr + k + 1];
    const uint32_t hb = in0 ^ ((in0 >> 1) | (in1 << 31));          // bottom side of cell I
    const uint32_t vb = in0 ^ up;                                  // left side
    const uint32_t vr = (vb >> 1) | ((in1 ^ up1) << 31);           // right side
    const uint32_t ht = up ^ ((up >> 1) | (up1 << 31));            // top side
    uint32_t active = hb | vb | vr | ht;
    while (active) {
        const int b = __ffs(active) - 1;
        active &= active - 1u;
        const int I = 32 * k + b;
        // corners counter-clockwise: 0 (I,J), 1 (I+1,J), 2 (I+1,J+1), 3 (I,J+1)
        const uint32_t in_c0 = (in0 >> b) & 1u, in_c3 = (up >> b) & 1u;
        const uint32_t in_c1 = b < 31 ? (in0 >> (b + 1)) & 1u : in1 & 1u;
        const uint32_t in_c2 = b < 31 ? (up >> (b + 1)) & 1u : up1 & 1u;
        const float v0 = value_at(sg, c, I, J);
        const float v1 = value_at(sg, c, I + 1, J);
        const float v3 = value_at(sg, c, I, J + 1);
        const int64_t eb = 2 * ((int64_t)J * c.W + I);
        if ((hb >> b) & 1u) {   // vertex on the bottom edge (I, J) -> (I+1, J)
            const uint32_t id = D.id(layer, I, J, 0);
            const float sa = in_c0 ? v0 : v1, sbv = in_c0 ? v1 : v0;
            const float t = (sa - c.C) / (sa - sbv);
            const float xp = in_c0 ? ((float)I - 0.5f + t) : ((float)I + 0.5f - t);
            *reinterpret_cast<float2*>(&rec[id].x) =
                make_float2(c.fx0 + xp * c.fpx, c.fy0 + ((float)J - 0.5f) * c.fpx);
            rec[id].eid = (int32_t)eb;
        }
        if ((vb >> b) & 1u) {   // vertex on the left edge (I, J) -> (I, J+1)
            const uint32_t id = D.id(layer, I, J, 1);
            const float sa = in_c0 ? v0 : v3, sbv = in_c0 ? v3 : v0;
            const float t = (sa - c.C) / (sa - sbv);
            const float yp = in_c0 ? ((float)J - 0.5f + t) : ((float)J + 0.5f - t);
            *reinterpret_cast<float2*>(&rec[id].x) =
                make_float2(c.fx0 + ((float)I - 0.5f) * c.fpx, c.fy0 + yp * c.fpx);
            rec[id].eid = (int32_t)(eb + 1);
        }
        // successors. Side k runs from corner k to corner k+1; bit k of nxt is corner k+1.
        const uint32_t cs = in_c0 | (in_c1 << 1) | (in_c2 << 2) | (in_c3 << 3);
        const uint32_t nxt = ((cs >> 1) | (cs << 3)) & 0xfu;
        const uint32_t enter = cs & ~nxt & 0xfu;   // inside -> outside
        const uint32_t leave = ~cs & nxt & 0xfu;   // outside -> inside
        auto side = [&](int s) -> uint32_t {   // sides: 0 bottom, 1 right, 2 top, 3 left
            return s == 0 ? D.id(layer, I, J, 0)
                          : (s == 1 ? D.id(layer, I + 1, J, 1)
                                    : (s == 2 ? D.id(layer, I, J + 1, 0) : D.id(layer, I, J, 1)));
        };
        if (__popc(enter) == 1) {
            rec[side(__ffs(enter) - 1)].succ = side(__ffs(leave) - 1);
        } else if (enter) {
            const float v2 = value_at(sg, c, I + 1, J + 1);
            const bool joined = 0.25f * (v0 + v1 + v2 + v3) >= c.C;
            const int k0 = __ffs(enter) - 1, k1 = 31 - __clz(enter);
            rec[side(k0)].succ = side(joined ? ((k0 + 1) & 3) : ((k0 + 3) & 3));
            rec[side(k1)].succ = side(joined ? ((k1 + 1) & 3) : ((k1 + 3) & 3));
        }
    }
}

// pred[succ[i]] = i. Every crossing must have exactly one successor in range;
// anything else is reported through *status and nothing is written out of range.
__global__ void k_pred(const Xing* __restrict__ rec, int64_t n, uint32_t* __restrict__ pred,
                       uint32_t* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = rec[i].succ;
        if ((int64_t)s < n) pred[s] = (uint32_t)i;
        else atomicOr(status, ST_CAPACITY);
    }
}

// Local minima (pred > i < succ) into a compact list; packed[] cleared.
__global__ void k_candidates(const Xing* __restrict__ rec, const uint32_t* __restrict__ pred,
                             int64_t n, uint32_t* __restrict__ cand, uint32_t* __restrict__ n_cand,
                             int64_t* __restrict__ packed) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        bool is_min = false;
        if (i < n) {
            const uint32_t q = (uint32_t)i;
            is_min = pred[q] > q && rec[q].succ > q;
            packed[i] = 0;
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, is_min);
        uint32_t pos = 0;
        if (lane == 0 && ball) pos = atomicAdd(n_cand, (uint32_t)__popc(ball));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (is_min) cand[pos + __popc(ball & ((1u << lane) - 1u))] = (uint32_t)i;
    }
}

// Walk kernels: loops have very uneven lengths. A persistent grid (one wave)
// splits the candidate list into one contiguous range per block; inside the
// block, each lane takes its next candidate from a shared-memory counter as
// soon as its walk ends, so no lane waits for another's long loop.
struct WorkRange {
    int64_t begin, end;
};

__device__ __forceinline__ WorkRange block_range(int64_t nc) {
    const int64_t per = (nc + gridDim.x - 1) / gridDim.x;
    const int64_t b = (int64_t)blockIdx.x * per;
    return {b < nc ? b : nc, b + per < nc ? b + per : nc};
}

__global__ void k_heads(const Xing* __restrict__ rec, const uint32_t* __restrict__ cand,
                        const uint32_t* __restrict__ n_cand, int64_t n,
                        int64_t* __restrict__ packed, uint32_t* status) {
    __shared__ uint32_t s_next;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const WorkRange r = block_range(*n_cand);
    for (int64_t t = r.begin + atomicAdd(&s_next, 1u); t < r.end;
         t = r.begin + atomicAdd(&s_next, 1u)) {
        const uint32_t q = cand[t];
        uint32_t j = rec[q].succ;
        int64_t len = 1;
        bool head = true;
        while (j != q) {
            if (j < q) { head = false; break; }
            if ((int64_t)j >= n || len > n) {   // corrupt links: report, never loop forever
                atomicOr(status, ST_CAPACITY);
                head = false;
                break;
            }
            j = rec[j].succ;
            ++len;
        }
        if (head) packed[q] = ((int64_t)1 << 32) | len;
    }
}

__global__ void k_write(const Xing* __restrict__ rec, const uint32_t* __restrict__ cand,
                        const uint32_t* __restrict__ n_cand, const int64_t* __restrict__ packed,
                        const int64_t* __restrict__ scan, int64_t n,
                        int64_t* __restrict__ loop_off, float2* __restrict__ oxy,
                        int32_t* __restrict__ oeid) {
    __shared__ uint32_t s_next;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const WorkRange r = block_range(*n_cand);
    for (int64_t t = r.begin + atomicAdd(&s_next, 1u); t < r.end;
         t = r.begin + atomicAdd(&s_next, 1u)) {
        const uint32_t q = cand[t];
        const int64_t p = packed[q];
        if (p == 0) continue;
        const int64_t len = p & 0xffffffffLL;
        const int64_t loop = scan[q] >> 32;
        const int64_t voff = scan[q] & 0xffffffffLL;
        loop_off[loop] = voff;
        uint32_t j = q;
        for (int64_t k = 0; k < len && (int64_t)j < n; ++k) {
            const Xing x = rec[j];
            oxy[voff + k] = make_float2(x.x, x.y);
            if (oeid) oeid[voff + k] = x.eid;
            j = x.succ;
        }
    }
}

int persistent_blocks(const void* kernel, int block) {
    int dev = 0, sms = 0, per_sm = 0;
    CSL_CUDA(cudaGetDevice(&dev));
    CSL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CSL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0));
    return std::max(1, sms * std::max(1, per_sm));
}

// layer_loops[l] = loops whose head lies before the first crossing of layer l
__global__ void k_layer_loops(const uint32_t* __restrict__ prefix, int64_t edge_wpl, int n_layers,
                              const int64_t* __restrict__ scan, int64_t n_cross, int64_t n_loops,
                              int64_t* __restrict__ layer_loops, int64_t* __restrict__ loop_off) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > n_layers) return;
    int64_t first = l < n_layers ? (int64_t)prefix[(int64_t)l * edge_wpl] : n_cross;
    layer_loops[l] = first < n_cross ? (scan[first] >> 32) : n_loops;
    if (l == 0) loop_off[n_loops] = n_cross;
}

}  // namespace

void contours_chunk(const ChunkGeom& g, double C, const float* sigma, const uint32_t* mask,
                    bool want_eid, ChunkContours& out, cudaStream_t s) {
    MsConst c;
    c.nx = g.nx;
    c.ny = g.ny;
    c.W = g.nx + 2;
    c.H = g.ny + 2;
    c.mwr = (int32_t)mask_words_per_row(g.nx);
    c.ewr = 2 * c.mwr;
    c.mask_wpl = mask_words_per_layer(g.nx, g.ny);
    c.edge_wpl = 2 * c.mask_wpl;
    c.n_layers = g.n_layers;
    c.C = (float)C;
    c.fx0 = (float)g.x0;
    c.fy0 = (float)g.y0;
    c.fpx = (float)g.px;
    const int64_t n_words = c.edge_wpl * g.n_layers;
    // 32-bit crossing ids: fewer than 2^27 edge words keeps every count below 2^32
    if (n_words >= ((int64_t)1 << 27)) fail(CSL_ERR_CAPACITY, "marching squares: chunk too large");

    DevBuf ew((size_t)n_words * 4, s), prefix((size_t)n_words * 4, s), total(8, s);
    {
        const int64_t n_thr = (int64_t)c.H * c.mwr;
        dim3 grid((unsigned)ceil_div(n_thr, 256), (unsigned)g.n_layers);
        k_edge_words<<<grid, 256, 0, s>>>(mask, c, ew.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms edge words");
    }
    k_popc<<<grid_for(n_words, 256), 256, 0, s>>>(ew.as<uint32_t>(), n_words, prefix.as<uint32_t>());
    CSL_LAUNCH_CHECK("ms popc");
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
    DevBuf rec((size_t)n_cross * sizeof(Xing), s);
    CSL_CUDA(cudaMemsetAsync(rec.get(), 0xff, (size_t)n_cross * sizeof(Xing), s));
    Dense D{ew.as<uint32_t>(), prefix.as<uint32_t>(), c.edge_wpl, c.ewr};
    {
        const int64_t n_thr = (int64_t)(c.ny + 1) * c.mwr;
        dim3 grid((unsigned)ceil_div(n_thr, 256), (unsigned)g.n_layers);
        k_emit<<<grid, 256, 0, s>>>(sigma, mask, c, D, rec.as<Xing>());
        CSL_LAUNCH_CHECK("ms emit");
    }
    DevBuf pred((size_t)n_cross * 4, s), cand((size_t)n_cross * 4, s);
    DevBuf packed((size_t)n_cross * 8, s), scan((size_t)n_cross * 8, s);
    DevBuf small(8, s);   // [0] status, [1] candidate count
    uint32_t* status = small.as<uint32_t>();
    uint32_t* n_cand = small.as<uint32_t>() + 1;
    CSL_CUDA(cudaMemsetAsync(small.get(), 0, 8, s));
    CSL_CUDA(cudaMemsetAsync(pred.get(), 0xff, (size_t)n_cross * 4, s));
    const unsigned gx = grid_for(n_cross, 256);
    k_pred<<<gx, 256, 0, s>>>(rec.as<Xing>(), n_cross, pred.as<uint32_t>(), status);
    CSL_LAUNCH_CHECK("ms pred");
    k_candidates<<<gx, 256, 0, s>>>(rec.as<Xing>(), pred.as<uint32_t>(), n_cross,
                                    cand.as<uint32_t>(), n_cand, packed.as<int64_t>());
    CSL_LAUNCH_CHECK("ms candidates");
    static int heads_blocks = persistent_blocks((const void*)k_heads, 256);
    static int write_blocks = persistent_blocks((const void*)k_write, 256);
    k_heads<<<heads_blocks, 256, 0, s>>>(rec.as<Xing>(), cand.as<uint32_t>(), n_cand, n_cross,
                                         packed.as<int64_t>(), status);
    CSL_LAUNCH_CHECK("ms heads");
    DevBuf tot(8, s);
    exclusive_scan_i64(packed.as<int64_t>(), scan.as<int64_t>(), n_cross, tot.as<int64_t>(), s);
    const int64_t packed_total = read_i64(tot.as<int64_t>(), s);
    uint32_t st = 0;
    read_to_host(&st, status, 4, s);
    if (st) fail(CSL_ERR_CUDA, "marching squares: inconsistent successor links");
    const int64_t n_loops = packed_total >> 32;
    if ((packed_total & 0xffffffffLL) != n_cross)
        fail(CSL_ERR_CUDA, "marching squares: loops do not cover every crossing");
    out.n_loops = n_loops;
    out.loop_off.ensure((size_t)(n_loops + 1) * 8, s);
    out.xy.ensure((size_t)n_cross * 8, s);
    if (want_eid) out.eid.ensure((size_t)n_cross * 4, s);
    k_write<<<write_blocks, 256, 0, s>>>(rec.as<Xing>(), cand.as<uint32_t>(), n_cand,
                                         packed.as<int64_t>(),
                                         scan.as<int64_t>(), n_cross, out.loop_off.as<int64_t>(),
                                         out.xy.as<float2>(),
                                         want_eid ? out.eid.as<int32_t>() : nullptr);
    CSL_LAUNCH_CHECK("ms write");
    k_layer_loops<<<(unsigned)ceil_div(g.n_layers + 1, 128), 128, 0, s>>>(
        prefix.as<uint32_t>(), c.edge_wpl, g.n_layers, scan.as<int64_t>(), n_cross, n_loops,
        out.layer_loops.as<int64_t>(), out.loop_off.as<int64_t>());
    CSL_LAUNCH_CHECK("ms layer loops");
}

}  // namespace csl
