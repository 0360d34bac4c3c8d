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
//   4. the head of a loop is its smallest id, which is a local minimum
//      (pred > id < succ). Splitters = all local minima plus a hashed 1-in-32
//      sample of crossings; each splitter walks its segment to the next
//      splitter, so no thread walks a whole long loop;
//   5. on the graph of splitters (one cycle per loop), a cycle of at most 16
//      splitters (every small loop) is resolved by walking it; on the rest,
//      pointer jumping gives every splitter its cycle's minimum (the head)
//      and, with the cycles cut before their heads, weighted list ranking
//      gives every segment its distance from the head;
//   6. a prefix sum over the heads (loop length) numbers the loops in head
//      order and places them; every splitter writes its segment there.
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

// grid: x over (row J, mask word k), y = layer. cnt: the crossings of each
// edge word (the input of the numbering scan).
__global__ void k_edge_words(const uint32_t* __restrict__ mask, MsConst c,
                             uint32_t* __restrict__ ew, uint32_t* __restrict__ cnt) {
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
    const int64_t row = (int64_t)layer * c.edge_wpl + (int64_t)J * c.ewr;
    reinterpret_cast<uint2*>(ew + row)[k] = out;
    reinterpret_cast<uint2*>(cnt + row)[k] = make_uint2(__popc(out.x), __popc(out.y));
}

// Crossing numbering: the crossing on the edge with bit `bit` of edge word w
// has id prefix[w] + popc(ew[w] & ((1 << bit) - 1)).
struct Dense {
    const uint32_t* ew;
    const uint32_t* prefix;
    int64_t edge_wpl;
    int32_t ewr;
};

// The fused pass's vertex lists (FusedVerts, as the field kernel leaves them).
struct FusedIn {
    const uint32_t* tbase;
    const uint16_t* roff;
    const float2* verts;
    const uint32_t* saddle;
    int32_t T, ntx, n_tiles;
};

// Vertex of the crossing on the edge from padded sample (I, J) in direction
// dir (0: x, 1: y): the tile owning the sample lists its crossings in edge-id
// order, so its place is the tile's base + the row's offset + the number of
// crossing edges of row J from the row's first owned sample up to this edge
// (the interleaved edge words hold exactly those bits).
__device__ __forceinline__ float2 fused_vertex(const FusedIn& F, const Dense& D, int layer, int I,
                                               int J, int dir) {
    const int tx = I == 0 ? 0 : (I - 1) / F.T, ty = J == 0 ? 0 : (J - 1) / F.T;
    const int b = J - 1 - ty * F.T;                 // tile-local row, -1 .. T - 1
    const int Ia = tx == 0 ? 0 : tx * F.T + 1;      // first sample of the row the tile owns
    const uint32_t* row = D.ew + (int64_t)layer * D.edge_wpl + (int64_t)J * D.ewr;
    const int lo = 2 * Ia, hi = 2 * I + dir;
    uint32_t rank = 0;
    for (int w = lo >> 5; w <= ((hi - 1) >> 5) && hi > lo; ++w) {
        uint32_t m = row[w];
        if (w == (lo >> 5)) m &= 0xffffffffu << (lo & 31);
        if (w == (hi >> 5)) m &= (1u << (hi & 31)) - 1u;
        rank += __popc(m);
    }
    const int64_t tl = (int64_t)layer * F.n_tiles + (int64_t)ty * F.ntx + tx;
    return F.verts[(int64_t)F.tbase[tl] + F.roff[tl * (F.T + 1) + b + 1] + rank];
}


// A block of k_emit covers a band of kEmitRows cell rows and kEmitWords mask
// words (32 cells each) of one layer: one thread per (row, word). The Sigma
// values its vertices and saddles need (pixel rows J0 - 1 .. J0 + kEmitRows - 1,
// columns 32 k0 - 1 .. 32 (k0 + kEmitWords) - 1) are staged into shared memory
// first with coalesced loads, so that every Sigma row is read from DRAM about
// once instead of as scattered words at each crossing. A staged row has a
// pitch of kEmitPitch floats: pixel 32 k0 + c sits at column 4 + c (16-byte
// aligned, so a thread moves 4 pixels with one vector load and store), pixel
// 32 k0 - 1 at column 3.
constexpr int kEmitRows = 8, kEmitWords = 32;
constexpr int kEmitPitch = 32 * kEmitWords + 4;
static_assert(32 * kEmitWords == 4 * 256, "one 4-pixel vector per thread and row");

// grid: x over (band of kEmitRows rows J <= ny, segment of kEmitWords mask
// words), y = layer. FUSED: vertices and saddle decisions from the fused pass
// (F) instead of Sigma.
template <bool FUSED>
__global__ void __launch_bounds__(256, 6) k_emit(const float* __restrict__ sigma, const uint32_t* __restrict__ mask,
                       MsConst c, Dense D, FusedIn F, Xing* __restrict__ rec, uint32_t n_cap,
                       uint32_t* flag) {
    __shared__ __align__(16) float s_sig[FUSED ? 4 : (kEmitRows + 1) * kEmitPitch];
    const int layer = blockIdx.y;
    const int n_segs = (c.mwr + kEmitWords - 1) / kEmitWords;
    const int band = blockIdx.x / n_segs, seg = blockIdx.x - band * n_segs;
    const int J0 = band * kEmitRows, k0 = seg * kEmitWords;
    const int J = J0 + (int)(threadIdx.x / kEmitWords), k = k0 + (int)(threadIdx.x % kEmitWords);
    const uint32_t* m = mask + (int64_t)layer * c.mask_wpl;
    const float* sg = FUSED ? nullptr : sigma + (int64_t)layer * c.nx * c.ny;
    // this thread's mask words, edge words and prefix sums (of its row, the
    // next word and the row above), loaded before the staging so that their
    // latency overlaps it; the other prefixes follow from these
    const bool live = J <= c.ny && k < c.mwr;
    const bool last = k + 1 >= c.mwr;
    uint32_t in0 = 0u, in1 = 0u, up = 0u, up1 = 0u;
    uint32_t e0 = 0u, e1 = 0u, e2 = 0u, p0 = 0u, u0 = 0u, u1 = 0u, q0 = 0u;
    if (live) {
        in0 = m[(int64_t)J * c.mwr + k];
        in1 = last ? 0u : m[(int64_t)J * c.mwr + k + 1];
        up = m[(int64_t)(J + 1) * c.mwr + k];          // J + 1 <= ny + 1 < H
        up1 = last ? 0u : m[(int64_t)(J + 1) * c.mwr + k + 1];
        const int64_t wb = layer * D.edge_wpl + (int64_t)J * D.ewr + 2 * k;
        const int64_t wu = wb + D.ewr;
        e0 = D.ew[wb];
        e1 = D.ew[wb + 1];
        e2 = last ? 0u : D.ew[wb + 2];
        p0 = D.prefix[wb];
        u0 = D.ew[wu];
        u1 = D.ew[wu + 1];
        q0 = D.prefix[wu];
    }
    if (!FUSED) {   // pixel (i, j) -> s_sig[(j - (J0 - 1)) * kEmitPitch + 4 + i - 32 k0]
        const int ib = 32 * k0 + 4 * (int)threadIdx.x;   // this thread's 4 pixels of each row
        // whole vectors need 16-byte aligned rows (nx % 4 == 0) and 4 pixels inside
        const bool vec = (c.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(sg) & 15) == 0 &&
                         ib + 3 < c.nx;
#pragma unroll
        for (int r = 0; r < kEmitRows + 1; ++r) {
            const int j = J0 - 1 + r;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (j >= 0 && j < c.ny) {
                const float* row = sg + (int64_t)j * c.nx;
                if (vec) {
                    v = __ldg(reinterpret_cast<const float4*>(row + ib));
                } else {
                    if (ib < c.nx) v.x = row[ib];
                    if (ib + 1 < c.nx) v.y = row[ib + 1];
                    if (ib + 2 < c.nx) v.z = row[ib + 2];
                    if (ib + 3 < c.nx) v.w = row[ib + 3];
                }
                if (threadIdx.x == 0)   // the pixel left of the band (column 3)
                    s_sig[r * kEmitPitch + 3] = (k0 > 0 && 32 * k0 - 1 < c.nx) ? row[32 * k0 - 1]
                                                                              : 0.0f;
            } else if (threadIdx.x == 0) {
                s_sig[r * kEmitPitch + 3] = 0.0f;
            }
            *reinterpret_cast<float4*>(&s_sig[r * kEmitPitch + 4 + 4 * threadIdx.x]) = v;
        }
        __syncthreads();
    }
    // Sigma at padded sample (I, J) of this block (0 outside the grid, like the ring)
    auto value_s = [&](int I, int J2) -> float {
        return s_sig[(J2 - J0) * kEmitPitch + (I - 32 * k0) + 3];
    };
    if (!live) return;
    const uint32_t hb = in0 ^ ((in0 >> 1) | (in1 << 31));          // bottom side of cell I
    const uint32_t vb = in0 ^ up;                                  // left side
    const uint32_t vr = (vb >> 1) | ((in1 ^ up1) << 31);           // right side
    const uint32_t ht = up ^ ((up >> 1) | (up1 << 31));            // top side
    uint32_t active = hb | vb | vr | ht;
    if (!active) return;
    // the prefix of a word is its left neighbour's plus that word's crossings:
    // every crossing id below comes from registers
    const uint32_t p1 = p0 + __popc(e0), p2 = last ? 0u : p1 + __popc(e1);
    const uint32_t q1 = q0 + __popc(u0);
    while (active) {
        const int b = __ffs(active) - 1;
        active &= active - 1u;
        const int I = 32 * k + b;
        // corners counter-clockwise: 0 (I,J), 1 (I+1,J), 2 (I+1,J+1), 3 (I,J+1)
        const uint32_t in_c0 = (in0 >> b) & 1u, in_c3 = (up >> b) & 1u;
        const uint32_t in_c1 = b < 31 ? (in0 >> (b + 1)) & 1u : in1 & 1u;
        const uint32_t in_c2 = b < 31 ? (up >> (b + 1)) & 1u : up1 & 1u;
        // ids of the crossings on the cell's sides (valid where the side crosses):
        // in the interleaved edge words, sample si's h edge is bit 2 (si % 16) and
        // its v edge the next bit; the right side is sample b + 1's v edge, the
        // top side the h edge of sample b in the row above
        const int bit = 2 * (b & 15);
        const uint32_t eb_w = b < 16 ? e0 : e1, pb_w = b < 16 ? p0 : p1;
        const uint32_t id_bottom = pb_w + __popc(eb_w & ((1u << bit) - 1u));
        const uint32_t id_left = id_bottom + ((eb_w >> bit) & 1u);
        const int sr = b + 1, bit_r = 2 * (sr & 15) + 1;
        const uint32_t er_w = sr < 16 ? e0 : (sr < 32 ? e1 : e2);
        const uint32_t pr_w = sr < 16 ? p0 : (sr < 32 ? p1 : p2);
        const uint32_t id_right = pr_w + __popc(er_w & ((1u << bit_r) - 1u));
        const uint32_t id_top = (b < 16 ? q0 : q1) + __popc((b < 16 ? u0 : u1) & ((1u << bit) - 1u));
        auto side = [&](int sd) -> uint32_t {   // sides: 0 bottom, 1 right, 2 top, 3 left
            return sd == 0 ? id_bottom : (sd == 1 ? id_right : (sd == 2 ? id_top : id_left));
        };
        const bool h_own = (hb >> b) & 1u, v_own = (vb >> b) & 1u;
        // Sigma only where a vertex is placed (or a saddle is decided)
        const float v0 = (!FUSED && (h_own || v_own)) ? value_s(I, J) : 0.0f;
        const int64_t eb = 2 * ((int64_t)J * c.W + I);
        if (h_own) {   // vertex on the bottom edge (I, J) -> (I+1, J)
            const uint32_t id = id_bottom;
            if (id >= n_cap) { atomicOr(flag, 1u); continue; }
            float2 xy;
            if (FUSED) {
                xy = fused_vertex(F, D, layer, I, J, 0);
            } else {
                const float v1 = value_s(I + 1, J);
                const float sa = in_c0 ? v0 : v1, sbv = in_c0 ? v1 : v0;
                const float t = __fdividef(sa - c.C, sa - sbv);   // in [0, 1]; sa > C > sbv
                const float xp = in_c0 ? ((float)I - 0.5f + t) : ((float)I + 0.5f - t);
                xy = make_float2(c.fx0 + xp * c.fpx, c.fy0 + ((float)J - 0.5f) * c.fpx);
            }
            *reinterpret_cast<float2*>(&rec[id].x) = xy;
            rec[id].eid = (int32_t)eb;
        }
        if (v_own) {   // vertex on the left edge (I, J) -> (I, J+1)
            const uint32_t id = id_left;
            if (id >= n_cap) { atomicOr(flag, 1u); continue; }
            float2 xy;
            if (FUSED) {
                xy = fused_vertex(F, D, layer, I, J, 1);
            } else {
                const float v3 = value_s(I, J + 1);
                const float sa = in_c0 ? v0 : v3, sbv = in_c0 ? v3 : v0;
                const float t = __fdividef(sa - c.C, sa - sbv);   // in [0, 1]; sa > C > sbv
                const float yp = in_c0 ? ((float)J - 0.5f + t) : ((float)J + 0.5f - t);
                xy = make_float2(c.fx0 + ((float)I - 0.5f) * c.fpx, c.fy0 + yp * c.fpx);
            }
            *reinterpret_cast<float2*>(&rec[id].x) = xy;
            rec[id].eid = (int32_t)(eb + 1);
        }
        // successors. Side k runs from corner k to corner k+1; bit k of nxt is corner k+1.
        const uint32_t cs = in_c0 | (in_c1 << 1) | (in_c2 << 2) | (in_c3 << 3);
        const uint32_t nxt = ((cs >> 1) | (cs << 3)) & 0xfu;
        const uint32_t enter = cs & ~nxt & 0xfu;   // inside -> outside
        const uint32_t leave = ~cs & nxt & 0xfu;   // outside -> inside
        if (__popc(enter) == 1) {
            const uint32_t a = side(__ffs(enter) - 1);
            if (a < n_cap) rec[a].succ = side(__ffs(leave) - 1);
            else atomicOr(flag, 1u);
        } else if (enter) {
            bool joined;
            if (FUSED) {
                const uint32_t sw = F.saddle[(int64_t)layer * c.mask_wpl + (int64_t)J * c.mwr +
                                             (I >> 5)];
                joined = (sw >> (I & 31)) & 1u;
            } else {
                const float w0 = value_s(I, J), w1 = value_s(I + 1, J);
                const float w2 = value_s(I + 1, J + 1), w3 = value_s(I, J + 1);
                joined = 0.25f * (w0 + w1 + w2 + w3) >= c.C;
            }
            const int k0 = __ffs(enter) - 1, k1 = 31 - __clz(enter);
            const uint32_t a0 = side(k0), a1 = side(k1);
            if (a0 < n_cap && a1 < n_cap) {
                rec[a0].succ = side(joined ? ((k0 + 1) & 3) : ((k0 + 3) & 3));
                rec[a1].succ = side(joined ? ((k1 + 1) & 3) : ((k1 + 3) & 3));
            } else {
                atomicOr(flag, 1u);
            }
        }
    }
}

// Splitters cut every loop into short segments: every local minimum
// (pred > id < succ; the loop's smallest id is one) and a hashed 1-in-32
// sample, so that a smooth loop with a single local minimum is cut too.
__device__ __forceinline__ bool is_splitter(uint32_t i, uint32_t pred_i, uint32_t succ_i) {
    return (pred_i > i && succ_i > i) || ((i * 2654435761u) >> 27) == 0u;
}

// For the successor s of every crossing i (i is s's predecessor): nxt[s] =
// succ(s) | (s is a splitter) << 31, the only array the segment walks read
// and the one whose top bits number the splitters. Thread i reads its own
// successor and its successor's (records of one contour lie close together),
// so no separate predecessor array is built. A successor out of range is
// reported through *status and nothing is written for it. Every crossing is
// somebody's successor (the entry crossing of its exit cell), so every entry
// is written; in a replay whose sizes changed, entries left out keep the 0
// they were cleared to (no splitter).
__global__ void k_split_flags(const Xing* __restrict__ rec, int64_t n,
                              uint32_t* __restrict__ nxt, uint32_t* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q = rec[i].succ;
        if ((int64_t)q >= n) {
            atomicOr(status, ST_CAPACITY);
            continue;
        }
        const uint32_t sc = rec[q].succ;
        const bool sp = is_splitter(q, (uint32_t)i, sc);
        nxt[q] = (sc & 0x7fffffffu) | (sp ? 0x80000000u : 0u);
    }
}

// Each splitter walks its segment up to the next splitter (nxt: successor |
// splitter bit, one 4-byte load per step). A walk is a chain of dependent
// loads, so every thread advances kWalks walks of different segments in
// lockstep: their loads are independent and in flight together.
constexpr int kWalks = 1;

__global__ void k_segments(const uint32_t* __restrict__ nxt,
                           const uint32_t* __restrict__ spos, const uint32_t* __restrict__ split_id,
                           int64_t ns, int64_t n, uint32_t* __restrict__ seg_next,
                           uint32_t* __restrict__ seg_len, uint32_t* status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < ns;
         t0 += stride * kWalks) {
        uint32_t j[kWalks];
        int64_t len[kWalks];
        bool live[kWalks], bad[kWalks];
#pragma unroll
        for (int g = 0; g < kWalks; ++g) {
            const int64_t t = t0 + g * stride;
            live[g] = bad[g] = false;
            len[g] = 1;
            j[g] = 0;
            if (t >= ns) continue;
            const uint32_t s0 = split_id[t];
            if ((int64_t)s0 >= n) {   // a replay whose sizes changed (flagged): no walk
                bad[g] = true;
                continue;
            }
            j[g] = nxt[s0] & 0x7fffffffu;
            live[g] = true;
        }
        for (;;) {
            bool any = false;
            uint32_t v[kWalks];
#pragma unroll
            for (int g = 0; g < kWalks; ++g) {
                if (live[g] && ((int64_t)j[g] >= n || len[g] > n)) {   // corrupt links
                    live[g] = false;
                    bad[g] = true;
                }
                v[g] = live[g] ? nxt[j[g]] : 0u;
            }
#pragma unroll
            for (int g = 0; g < kWalks; ++g) {
                if (!live[g]) continue;
                if (v[g] >> 31) {   // the next splitter
                    live[g] = false;
                } else {
                    j[g] = v[g] & 0x7fffffffu;
                    ++len[g];
                    any = true;
                }
            }
            if (!any) break;
        }
#pragma unroll
        for (int g = 0; g < kWalks; ++g) {
            const int64_t t = t0 + g * stride;
            if (t >= ns) continue;
            uint32_t sn = 0;
            if (!bad[g]) {
                sn = spos[j[g]];
                if ((int64_t)sn >= ns) bad[g] = true;   // more splitters than planned (flagged)
            }
            if (bad[g]) {   // report, never loop forever
                atomicOr(status, ST_CAPACITY);
                seg_next[t] = (uint32_t)t;
                seg_len[t] = 1;
            } else {
                seg_next[t] = sn;
                seg_len[t] = (uint32_t)len[g];
            }
        }
    }
}

// One doubling step of the cycle minimum over the splitter graph:
// (cm, nx) -> (min(cm, cm[nx]), nx[nx]); sets done[it] when it changes cm.
// Once a step changed nothing, the later steps only copy cm forward, so the
// result is always in the buffer of the last step.
__global__ void k_jump_min(const uint32_t* __restrict__ cm, const uint32_t* __restrict__ nx,
                           uint32_t* __restrict__ cm2, uint32_t* __restrict__ nx2, int64_t ns,
                           uint32_t* done, int it) {
    if (it > 0 && done[it - 1] == 0) {   // converged: carry the result forward
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns;
             t += (int64_t)gridDim.x * blockDim.x)
            cm2[t] = cm[t];
        return;
    }
    bool changed = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cm[t];
        uint32_t nt = nx[t];
        if ((int64_t)nt >= ns) nt = (uint32_t)t;   // only in a flagged replay
        const uint32_t b = cm[nt];
        const uint32_t m = b < a ? b : a;
        changed |= m != a;
        cm2[t] = m;
        nx2[t] = nx[nt];
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) done[it] = 1u;
}

// One doubling step of weighted list ranking: dist += dist[nx], nx = nx[nx].
__global__ void k_jump_rank(const uint32_t* __restrict__ dist, const uint32_t* __restrict__ nx,
                            uint32_t* __restrict__ dist2, uint32_t* __restrict__ nx2, int64_t ns,
                            uint32_t* done, int it) {
    if (it > 0 && done[it - 1] == 0) {   // every list ended: carry the result forward
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns;
             t += (int64_t)gridDim.x * blockDim.x)
            dist2[t] = dist[t];
        return;
    }
    bool live = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t nt = nx[t];
        if ((int64_t)nt >= ns) {   // list end (or, in a flagged replay, a bad link)
            dist2[t] = dist[t];
            nx2[t] = nt;
        } else {
            dist2[t] = dist[t] + dist[nt];
            const uint32_t nn = nx[nt];
            nx2[t] = nn;
            live |= (int64_t)nn < ns;
        }
    }
    if (__syncthreads_or(live) && threadIdx.x == 0) done[it] = 1u;
}

// Splitter cycles of at most kShortCycle splitters (all the small loops) are
// resolved by walking them; the rest go to pointer jumping on a compact list.
constexpr int kShortCycle = 16;
constexpr uint32_t kNil = 0xffffffffu;

// cm[t] = the cycle's smallest splitter id when t's cycle closes within
// kShortCycle steps; otherwise t is appended to the long list. The head of a
// short cycle (the splitter holding its smallest id) then walks it once more:
// rank_start = crossings of the loop before each segment, loop_len at the head.
__global__ void k_short_cycles(const uint32_t* __restrict__ split_id,
                               const uint32_t* __restrict__ seg_next,
                               const uint32_t* __restrict__ seg_len, int64_t ns,
                               uint32_t* __restrict__ cm, uint32_t* __restrict__ long_list,
                               uint32_t* __restrict__ long_pos, uint32_t* __restrict__ n_long,
                               uint32_t* __restrict__ rank_start,
                               uint32_t* __restrict__ loop_len) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ns;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        bool is_long = false;
        if (t < ns) {
            uint32_t v = seg_next[t], mn = split_id[t];
            int n = 1;
            while (v != (uint32_t)t && n < kShortCycle) {
                const uint32_t id = split_id[v];
                mn = id < mn ? id : mn;
                v = seg_next[v];
                ++n;
            }
            is_long = v != (uint32_t)t;
            cm[t] = is_long ? kNil : mn;
            long_pos[t] = kNil;
            if (!is_long && mn == split_id[t]) {   // the head: rank the cycle's segments
                uint32_t acc = 0, w = (uint32_t)t;
                int m = 0;
                do {
                    rank_start[w] = acc;
                    acc += seg_len[w];
                    w = seg_next[w];
                } while (w != (uint32_t)t && ++m < kShortCycle);
                loop_len[t] = acc;
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, is_long);
        uint32_t pos = 0;
        if (lane == 0 && ball) pos = atomicAdd(n_long, (uint32_t)__popc(ball));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (is_long) {
            const uint32_t q = pos + __popc(ball & ((1u << lane) - 1u));
            long_list[q] = (uint32_t)t;
            long_pos[t] = q;
        }
    }
}

// Compact long-cycle graph: node u = long_list[u]; next in compact indices.
__global__ void k_long_setup(const uint32_t* __restrict__ long_list,
                             const uint32_t* __restrict__ long_pos,
                             const uint32_t* __restrict__ split_id,
                             const uint32_t* __restrict__ seg_next, int64_t nl,
                             uint32_t* __restrict__ lcm, uint32_t* __restrict__ lnx) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nl;
         u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = long_list[u];
        const uint32_t nt = seg_next[t];   // < ns by construction of k_segments
        lcm[u] = split_id[t];
        lnx[u] = long_pos[nt];
    }
}

// Break each long cycle before its head (nx = NIL there); dist = segment length.
__global__ void k_long_break(const uint32_t* __restrict__ lcm, const uint32_t* __restrict__ long_list,
                             const uint32_t* __restrict__ long_pos,
                             const uint32_t* __restrict__ split_id,
                             const uint32_t* __restrict__ seg_next,
                             const uint32_t* __restrict__ seg_len, int64_t nl,
                             uint32_t* __restrict__ nx, uint32_t* __restrict__ dist) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nl;
         u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = long_list[u];
        const uint32_t nt = seg_next[t];
        const uint32_t nu = long_pos[nt];
        nx[u] = ((int64_t)nu >= nl || lcm[nu] == split_id[nt]) ? kNil : nu;
        dist[u] = seg_len[t];
    }
}

// Back to splitter order: cm, rank_start = loop length - dist, loop_len at heads.
__global__ void k_long_ranks(const uint32_t* __restrict__ lcm, const uint32_t* __restrict__ dist,
                             const uint32_t* __restrict__ long_list,
                             const uint32_t* __restrict__ long_pos,
                             const uint32_t* __restrict__ spos, int64_t nl, int64_t ns,
                             uint32_t* __restrict__ cm, uint32_t* __restrict__ rank_start,
                             uint32_t* __restrict__ loop_len) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nl;
         u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = long_list[u];
        const uint32_t sp = spos[lcm[u]];
        uint32_t hu = (int64_t)sp < ns ? long_pos[sp] : kNil;
        if ((int64_t)hu >= nl) hu = (uint32_t)u;   // only in a flagged replay
        cm[t] = lcm[u];
        rank_start[t] = dist[hu] - dist[u];
        if (hu == (uint32_t)u) loop_len[t] = dist[u];
    }
}

// packed[t] = (1 << 32) | loop length for heads, else 0 (splitter order).
__global__ void k_head_flags(const uint32_t* __restrict__ cm, const uint32_t* __restrict__ split_id,
                             const uint32_t* __restrict__ loop_len, int64_t ns,
                             int64_t* __restrict__ packed) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns;
         t += (int64_t)gridDim.x * blockDim.x)
        packed[t] = cm[t] == split_id[t] ? (((int64_t)1 << 32) | loop_len[t]) : 0;
}

// Replay checks: a device count against the planned one, and the status word.
__global__ void k_check_u32(const uint32_t* __restrict__ v, uint32_t expect, uint32_t* flag) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *v != expect) atomicOr(flag, 1u);
}
__global__ void k_check_packed(const int64_t* __restrict__ total, int64_t n_loops, int64_t n_cross,
                               const uint32_t* __restrict__ status, uint32_t* flag) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if ((*total >> 32) != n_loops || (*total & 0xffffffffLL) != n_cross) atomicOr(flag, 1u);
    if (*status) atomicOr(flag, 2u);
}

// Each splitter writes its segment at its loop's offset + rank_start; as in
// k_segments, every thread walks kWalks segments in lockstep. (Following the
// 4-byte successor array instead, with the records loaded beside the chain,
// measured no faster: a step then reads two sectors instead of one.)
__global__ void k_write_segments(const Xing* __restrict__ rec, const uint32_t* __restrict__ cm,
                                 const uint32_t* __restrict__ spos,
                                 const uint32_t* __restrict__ split_id,
                                 const uint32_t* __restrict__ seg_len,
                                 const uint32_t* __restrict__ rank_start,
                                 const int64_t* __restrict__ scan, int64_t ns, int64_t n,
                                 int64_t n_loops, int64_t vofs, int64_t* __restrict__ loop_off,
                                 float2* __restrict__ oxy, int32_t* __restrict__ oeid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < ns;
         t0 += stride * kWalks) {
        uint32_t j[kWalks];
        int64_t base[kWalks], len[kWalks];
        int64_t max_len = 0;
#pragma unroll
        for (int g = 0; g < kWalks; ++g) {
            const int64_t t = t0 + g * stride;
            len[g] = 0;
            base[g] = 0;
            j[g] = 0;
            if (t >= ns) continue;
            const uint32_t ht = cm[t];
            if ((int64_t)ht >= n) continue;              // only if the links were inconsistent
            const uint32_t h = spos[ht];                 // the head splitter of this loop
            if ((int64_t)h >= ns) continue;
            const int64_t voff = scan[h] & 0xffffffffLL;
            if (h == (uint32_t)t && (scan[h] >> 32) < n_loops) loop_off[scan[h] >> 32] = vofs + voff;
            const int64_t b = voff + (int64_t)rank_start[t];
            const int64_t l = seg_len[t];
            if (b < 0 || b + l > n) continue;           // only if the links were inconsistent
            base[g] = b;
            len[g] = l;
            j[g] = split_id[t];
            max_len = max(max_len, l);
        }
        for (int64_t r = 0; r < max_len; ++r) {
            Xing x[kWalks];
#pragma unroll
            for (int g = 0; g < kWalks; ++g)
                if (r < len[g] && (int64_t)j[g] < n) x[g] = rec[j[g]];
#pragma unroll
            for (int g = 0; g < kWalks; ++g) {
                if (r < len[g] && (int64_t)j[g] < n) {
                    oxy[base[g] + r] = make_float2(x[g].x, x[g].y);
                    if (oeid) oeid[base[g] + r] = x[g].eid;
                    j[g] = x[g].succ;
                }
            }
        }
    }
}

// layer_loops[l] = loops whose head lies before the first crossing of layer l
// (+ lofs); the chunk's closing vertex offset (+ vofs)
__global__ void k_layer_loops(const uint32_t* __restrict__ prefix, int64_t edge_wpl, int n_layers,
                              const uint32_t* __restrict__ spos, const int64_t* __restrict__ scan,
                              int64_t n_cross, int64_t ns, int64_t n_loops, int64_t lofs,
                              int64_t vofs, int64_t* __restrict__ layer_loops,
                              int64_t* __restrict__ loop_off) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > n_layers) return;
    const int64_t first = l < n_layers ? (int64_t)prefix[(int64_t)l * edge_wpl] : n_cross;
    const int64_t sp = first < n_cross ? (int64_t)spos[first] : ns;
    layer_loops[l] = lofs + (sp < ns ? (scan[sp] >> 32) : n_loops);
    if (l == 0) loop_off[n_loops] = vofs + n_cross;
}

__global__ void k_fill_i64(int64_t* __restrict__ a, int64_t n, int64_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace

void contours_chunk(const ChunkGeom& g, double C, const float* sigma, const uint32_t* mask,
                    bool want_eid, ChunkContours& out, cudaStream_t s, const Replay* rp,
                    const FusedVerts* fv, const ChunkDest* dest) {
    const bool replay = rp && rp->replay;
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

    // small: [0] status, [1] crossings, [2] splitters, [3..66] done, [67] long count
    DevBuf small(4 * 80, s);
    CSL_CUDA(cudaMemsetAsync(small.get(), 0, 4 * 80, s));
    uint32_t* status = small.as<uint32_t>();
    uint32_t* done = small.as<uint32_t>() + 3;
    uint32_t* n_long = small.as<uint32_t>() + 67;
    uint32_t* flag = rp ? rp->flag : status;   // where replay mismatches go

    DevBuf ew((size_t)n_words * 4, s), prefix((size_t)n_words * 4, s);
    {
        const int64_t n_thr = (int64_t)c.H * c.mwr;
        dim3 grid((unsigned)ceil_div(n_thr, 256), (unsigned)g.n_layers);
        k_edge_words<<<grid, 256, 0, s>>>(mask, c, ew.as<uint32_t>(), prefix.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms edge words");
    }
    exclusive_scan_u32(prefix.as<uint32_t>(), prefix.as<uint32_t>(), n_words, status + 1, s);
    int64_t n_cross;
    if (replay) {
        n_cross = rp->plan->n_cross;
        k_check_u32<<<1, 32, 0, s>>>(status + 1, (uint32_t)n_cross, flag);
        CSL_LAUNCH_CHECK("check crossings");
    } else {
        uint32_t v = 0;
        read_to_host(&v, status + 1, 4, s);
        n_cross = v;
        if (rp) rp->plan->n_cross = n_cross;
    }
    out.n_verts = n_cross;
    out.layer_loops.ensure((size_t)(g.n_layers + 1) * 8, s);
    if (n_cross == 0) {
        out.n_loops = 0;
        if (dest) {   // no loops: every layer starts at the running loop count
            dest->make_room(dest->v_base, dest->l_base + 1);
            k_fill_i64<<<1, 128, 0, s>>>(out.layer_loops.as<int64_t>(), g.n_layers + 1,
                                         dest->l_base);
            CSL_LAUNCH_CHECK("ms empty layers");
            k_fill_i64<<<1, 32, 0, s>>>(dest->loop_off + dest->l_base, 1, dest->v_base);
            CSL_LAUNCH_CHECK("ms empty chunk");
        } else {
            CSL_CUDA(cudaMemsetAsync(out.layer_loops.get(), 0, (size_t)(g.n_layers + 1) * 8, s));
            out.loop_off.ensure(8, s);
            CSL_CUDA(cudaMemsetAsync(out.loop_off.get(), 0, 8, s));
        }
        if (rp && !replay) rp->plan->ns = rp->plan->nl = rp->plan->n_loops = 0;
        return;
    }
    // the successor bit trick of k_split_flags needs ids below 2^31
    if (n_cross >= ((int64_t)1 << 31)) fail(CSL_ERR_CAPACITY, "marching squares: too many crossings");
    DevBuf rec((size_t)n_cross * sizeof(Xing), s);
    // Every record is written whole by k_emit: x, y and the edge id by the cell
    // that owns the edge, the successor by the cell the contour enters through
    // it (each crossing edge is the entry side of exactly one of its two cells).
    // A replay (planned sizes) may leave records unwritten when its sizes
    // changed: there they start as invalid ids, so that no walk follows them.
    if (rp) CSL_CUDA(cudaMemsetAsync(rec.get(), 0xff, (size_t)n_cross * sizeof(Xing), s));

    Dense D{ew.as<uint32_t>(), prefix.as<uint32_t>(), c.edge_wpl, c.ewr};
    {
        const int64_t n_bands = ceil_div((int64_t)c.ny + 1, kEmitRows);
        const int64_t n_segs = ceil_div((int64_t)c.mwr, kEmitWords);
        dim3 grid((unsigned)(n_bands * n_segs), (unsigned)g.n_layers);
        FusedIn F{};
        if (fv) {
            F.tbase = fv->tbase.as<uint32_t>();
            F.roff = fv->roff.as<uint16_t>();
            F.verts = fv->verts.as<float2>();
            F.saddle = fv->saddle.as<uint32_t>();
            F.T = g.T;
            F.ntx = g.ntx;
            F.n_tiles = g.ntx * g.nty;
            k_emit<true><<<grid, 256, 0, s>>>(sigma, mask, c, D, F, rec.as<Xing>(),
                                              (uint32_t)n_cross, flag);
        } else {
            k_emit<false><<<grid, 256, 0, s>>>(sigma, mask, c, D, F, rec.as<Xing>(),
                                               (uint32_t)n_cross, flag);
        }
        CSL_LAUNCH_CHECK("ms emit");
    }
    // ---- loops: splitters, segments, pointer jumping on the splitter graph
    // nxt[i] = succ(i) | splitter << 31 (0 for a crossing nobody points to);
    // one scan over its top bits numbers the splitters (spos, for every
    // crossing) and lists them (split_id) in the same pass
    DevBuf spos((size_t)n_cross * 4, s), nxt((size_t)n_cross * 4, s);
    // every crossing is the successor of the crossing through which the
    // contour enters its cell, so every entry is written; a replay whose sizes
    // changed may leave some out: there they start as 0 (no splitter)
    if (rp) CSL_CUDA(cudaMemsetAsync(nxt.get(), 0, (size_t)n_cross * 4, s));
    const unsigned gx = grid_for(n_cross, 256);
    k_split_flags<<<gx, 256, 0, s>>>(rec.as<Xing>(), n_cross, nxt.as<uint32_t>(), status);
    CSL_LAUNCH_CHECK("ms splitter flags");
    // the list's room: every crossing, or a replay's planned count
    const int64_t ns_cap = replay ? rp->plan->ns : n_cross;
    DevBuf split_id((size_t)std::max<int64_t>(ns_cap, 1) * 4, s);
    // a replay whose sizes changed leaves entries unwritten: make them valid ids
    if (replay) CSL_CUDA(cudaMemsetAsync(split_id.get(), 0, (size_t)ns_cap * 4, s));
    scan_flags_list(nxt.as<uint32_t>(), n_cross, spos.as<uint32_t>(), split_id.as<uint32_t>(),
                    ns_cap, status + 2, status, s);
    int64_t ns;
    if (replay) {
        ns = rp->plan->ns;
        k_check_u32<<<1, 32, 0, s>>>(status + 2, (uint32_t)ns, flag);
        CSL_LAUNCH_CHECK("check splitters");
    } else {
        uint32_t head2[3];
        read_to_host(head2, small.get(), 12, s);
        if (head2[0]) fail(CSL_ERR_CUDA, "marching squares: a crossing has no successor");
        ns = head2[2];
        if (rp) rp->plan->ns = ns;
    }
    DevBuf seg_next((size_t)ns * 4, s), seg_len((size_t)ns * 4, s);
    const unsigned gs = grid_for(ns, 256);
    k_segments<<<gs, 256, 0, s>>>(nxt.as<uint32_t>(), spos.as<uint32_t>(),
                                  split_id.as<uint32_t>(), ns, n_cross, seg_next.as<uint32_t>(),
                                  seg_len.as<uint32_t>(), status);
    CSL_LAUNCH_CHECK("ms segments");
    nxt.release();
    // short splitter cycles by walking them; long ones by pointer jumping
    DevBuf cm((size_t)ns * 4, s), long_list((size_t)ns * 4, s), long_pos((size_t)ns * 4, s);
    DevBuf rank_start((size_t)ns * 4, s), loop_len((size_t)ns * 4, s);
    if (replay) CSL_CUDA(cudaMemsetAsync(long_list.get(), 0, (size_t)ns * 4, s));
    k_short_cycles<<<gs, 256, 0, s>>>(split_id.as<uint32_t>(), seg_next.as<uint32_t>(),
                                      seg_len.as<uint32_t>(), ns, cm.as<uint32_t>(),
                                      long_list.as<uint32_t>(), long_pos.as<uint32_t>(), n_long,
                                      rank_start.as<uint32_t>(), loop_len.as<uint32_t>());
    CSL_LAUNCH_CHECK("ms short cycles");
    int64_t nl;
    if (replay) {
        nl = rp->plan->nl;
        k_check_u32<<<1, 32, 0, s>>>(n_long, (uint32_t)nl, flag);
        CSL_LAUNCH_CHECK("check long cycles");
    } else {
        uint32_t v = 0;
        read_to_host(&v, n_long, 4, s);
        nl = v;
        if (rp) rp->plan->nl = nl;
    }
    if (nl > 0) {
        // cycle minimum by doubling (later steps copy the converged result forward)
        int max_it = 1;
        while (((int64_t)1 << max_it) < nl + 1) ++max_it;
        max_it += 1;
        if (max_it > 60) fail(CSL_ERR_CAPACITY, "marching squares: too many splitters");
        DevBuf cmA((size_t)nl * 4, s), cmB((size_t)nl * 4, s), nxA((size_t)nl * 4, s),
            nxB((size_t)nl * 4, s);
        const unsigned gl = grid_for(nl, 256);
        k_long_setup<<<gl, 256, 0, s>>>(long_list.as<uint32_t>(), long_pos.as<uint32_t>(),
                                        split_id.as<uint32_t>(), seg_next.as<uint32_t>(), nl,
                                        cmA.as<uint32_t>(), nxA.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms long setup");
        uint32_t *a_cm = cmA.as<uint32_t>(), *a_nx = nxA.as<uint32_t>();
        uint32_t *b_cm = cmB.as<uint32_t>(), *b_nx = nxB.as<uint32_t>();
        for (int it = 0; it < max_it; ++it) {
            k_jump_min<<<gl, 256, 0, s>>>(a_cm, a_nx, b_cm, b_nx, nl, done, it);
            CSL_LAUNCH_CHECK("ms cycle minimum");
            std::swap(a_cm, b_cm);
            std::swap(a_nx, b_nx);
        }
        uint32_t* lcm = a_cm;   // the buffer the last step wrote
        DevBuf dA((size_t)nl * 4, s), dB((size_t)nl * 4, s), nxr_buf((size_t)nl * 4, s);
        uint32_t *nxr = nxr_buf.as<uint32_t>(), *nxr2 = (lcm == cmA.as<uint32_t>())
                                                            ? cmB.as<uint32_t>()
                                                            : cmA.as<uint32_t>();
        k_long_break<<<gl, 256, 0, s>>>(lcm, long_list.as<uint32_t>(), long_pos.as<uint32_t>(),
                                        split_id.as<uint32_t>(), seg_next.as<uint32_t>(),
                                        seg_len.as<uint32_t>(), nl, nxr, dA.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms break cycles");
        CSL_CUDA(cudaMemsetAsync(done, 0, 4 * 64, s));
        uint32_t *dist = dA.as<uint32_t>(), *dist2 = dB.as<uint32_t>();
        for (int it = 0; it < max_it; ++it) {
            k_jump_rank<<<gl, 256, 0, s>>>(dist, nxr, dist2, nxr2, nl, done, it);
            CSL_LAUNCH_CHECK("ms list ranking");
            std::swap(dist, dist2);
            std::swap(nxr, nxr2);
        }
        k_long_ranks<<<gl, 256, 0, s>>>(lcm, dist, long_list.as<uint32_t>(),
                                        long_pos.as<uint32_t>(), spos.as<uint32_t>(), nl, ns,
                                        cm.as<uint32_t>(), rank_start.as<uint32_t>(),
                                        loop_len.as<uint32_t>());
        CSL_LAUNCH_CHECK("ms long ranks");
    }
    DevBuf packed((size_t)ns * 8, s), scan((size_t)ns * 8, s), tot(8, s);
    k_head_flags<<<gs, 256, 0, s>>>(cm.as<uint32_t>(), split_id.as<uint32_t>(),
                                    loop_len.as<uint32_t>(), ns, packed.as<int64_t>());
    CSL_LAUNCH_CHECK("ms heads");
    exclusive_scan_i64(packed.as<int64_t>(), scan.as<int64_t>(), ns, tot.as<int64_t>(), s);
    int64_t n_loops;
    if (replay) {
        n_loops = rp->plan->n_loops;
        k_check_packed<<<1, 32, 0, s>>>(tot.as<int64_t>(), n_loops, n_cross, status, flag);
        CSL_LAUNCH_CHECK("check loops");
    } else {
        const int64_t packed_total = read_i64(tot.as<int64_t>(), s);
        uint32_t st = 0;
        read_to_host(&st, status, 4, s);
        if (st) fail(CSL_ERR_CUDA, "marching squares: inconsistent successor links");
        n_loops = packed_total >> 32;
        if ((packed_total & 0xffffffffLL) != n_cross)
            fail(CSL_ERR_CUDA, "marching squares: loops do not cover every crossing");
        if (rp) rp->plan->n_loops = n_loops;
    }
    out.n_loops = n_loops;
    // where the vertices and loop offsets go: the chunk's own arrays, or the
    // caller's growing result at its running bases
    int64_t* o_loop;
    float2* o_xy;
    int32_t* o_eid;
    int64_t vofs = 0, lofs = 0;
    if (dest) {
        dest->make_room(dest->v_base + n_cross, dest->l_base + n_loops + 1);
        vofs = dest->v_base;
        lofs = dest->l_base;
        o_loop = dest->loop_off + lofs;
        o_xy = dest->xy + vofs;
        o_eid = want_eid ? dest->eid + vofs : nullptr;
    } else {
        out.loop_off.ensure((size_t)(n_loops + 1) * 8, s);
        out.xy.ensure((size_t)n_cross * 8, s);
        if (want_eid) out.eid.ensure((size_t)n_cross * 4, s);
        o_loop = out.loop_off.as<int64_t>();
        o_xy = out.xy.as<float2>();
        o_eid = want_eid ? out.eid.as<int32_t>() : nullptr;
    }
    // one thread per splitter, not a grid-stride loop over a capped grid: a
    // CTA retires as soon as its 256 walks are done (walk lengths vary), and
    // the walks in flight are those of consecutive splitters (100M workload:
    // contour stage 141 -> 132 ms against 64 CTAs per SM)
    const unsigned gw = (unsigned)std::max<int64_t>(ceil_div(ns, (int64_t)256), (int64_t)1);
    k_write_segments<<<gw, 256, 0, s>>>(rec.as<Xing>(), cm.as<uint32_t>(), spos.as<uint32_t>(),
                                        split_id.as<uint32_t>(), seg_len.as<uint32_t>(),
                                        rank_start.as<uint32_t>(), scan.as<int64_t>(), ns, n_cross,
                                        n_loops, vofs, o_loop, o_xy, o_eid);
    CSL_LAUNCH_CHECK("ms write");
    k_layer_loops<<<(unsigned)ceil_div(g.n_layers + 1, 128), 128, 0, s>>>(
        prefix.as<uint32_t>(), c.edge_wpl, g.n_layers, spos.as<uint32_t>(), scan.as<int64_t>(),
        n_cross, ns, n_loops, lofs, vofs, out.layer_loops.as<int64_t>(), o_loop);
    CSL_LAUNCH_CHECK("ms layer loops");
}

}  // namespace csl
