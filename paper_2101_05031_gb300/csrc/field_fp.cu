// Footprint field kernel: Sigma(p) = sum_j w_j I_j(p) (Eq. 6, the segment
// integral of Eq. 7 by 3-point Gauss-Legendre, as in field.cu) on a T x T
// tile of a slab of S layers, with the work organised by edge instead of by
// pixel block.
//
// One CTA per (tile, slab), one warp per layer of the slab. The tile's record
// list (contiguous, in list order) is staged into shared memory by TMA bulk
// copies, as in field.cu. For each record, the warp of layer l computes the
// record's footprint in the plane z_l: the pixels whose centres can lie
// within R of the edge. In the plane, the points within distance r of the
// edge's line form, on every pixel row y = Y (relative to v_s, Z = z_l - v_s^z,
// a = u_y^2 + u_z^2), the interval |X - X*| <= sqrt(r^2 a - (Z u_y - Y u_z)^2)
// / a around X* = u_x (Y u_y + Z u_z) / a (Lagrange's identity); its half
// width is at most r / sqrt(a), and X* is affine in the row index. The warp
// takes rows when |u_y| >= |u_x| (then a >= 1/2) and columns otherwise (the
// same with x and y exchanged), so the span is at most 2 sqrt(2) r wide. The
// footprint is the rows of the edge's clipped box (the edge cut to
// |z - z_l| <= R, its xy box grown by R), each with its span of width
// W = floor(2 r / (sqrt(a) px) + 0.1) + 1 starting at ceil((X* - r/sqrt(a)) /
// px - 0.55), clipped to the box and the tile. The warp's 32 lanes run over
// rows x span as one dense index range, evaluate the segment term at their
// pixel, and add w I into the layer's Sigma plane in shared memory. The
// pixels of one pass are distinct and a warp walks its records in list
// order, so every pixel receives its terms in list order: the sum is
// deterministic (the pixels a footprint leaves out have I = 0). Pixel
// coordinates are formed as affine functions of the pixel indices, and where
// the edge covers the whole chord of every reached pixel's sphere the term is
// the closed form (16/15) w^5 / R^4, so values agree with field.cu's within
// FP32 rounding rather than bit for bit. Edges of zero length (u = 0) take
// their clipped box.
//
// Compared with the 8 x 4-pixel warp blocks of field.cu, the lanes follow the
// shape of the support (an ellipse of semi-axes R and R / cos(tilt)), which
// pays where the support is a few pixels across; where it covers whole tiles
// the block kernel loses nothing and keeps its sums in registers.
#include <math.h>

#include "field_tile.cuh"
#include "slice.cuh"

namespace csl {
namespace {

struct FpConst {
    int32_t nx, ny, ntx, n_tiles;
    int32_t n_layers;    // layers in this chunk
    int32_t K;           // records staged per bulk copy
    float R2, inv_R4, fpx, inv_px, fdz, cull;
    float C;             // iso-value (inside mask)
    const float2* org_x; // per tile column: x of its first pixel edge, (hi, lo)
    const float2* org_y; // per tile row
    const float2* org_z; // per slab: z of its first layer
    int32_t mwr;         // mask words per row
    int64_t mask_wpl;    // mask words per layer
    uint32_t* err;       // device status word: ST_TIMEOUT when a wait gave up
};

// One (record, layer) footprint, 16 bytes: the span of row (or column) u
// starts at ceil(c0 + u c1); w1 = record (< 2^14) | interior << 14 | mode << 15
// | W << 16 | passes << 24,
// geom = u0 | n_rows << 8 | v0 << 16 | v1 << 24 (u: rows in row mode, v: the
// pixels along them, [v0, v1] the clipped box).
struct __align__(16) Foot {
    float c0, c1;
    uint32_t w1, geom;
};

// Footprint of record (A, B) in layer plane zl of a T x T tile; false when
// the edge's support misses the tile in that plane.
template <int T>
__device__ __forceinline__ bool make_foot(const float4 A, const float4 B, float zl, int rec,
                                          const FpConst& c, Foot& f) {
    const float ax = A.x, ay = A.y, az = A.z, ux = A.w, uy = B.x, uz = B.y, len = B.z;
    float t_lo = 0.0f, t_hi = len;
    bool interior = false;
    if (uz > 1e-12f) {
        // approximate reciprocal: its relative error (~1e-7) moves these bounds
        // by far less than the cull margin (cull - R >= 1e-6 mm)
        const float inv_uz = __fdividef(1.0f, uz);
        const float ta = (zl - c.cull - az) * inv_uz, tb = (zl + c.cull - az) * inv_uz;
        // every pixel within R of the line in this plane has t0 in (ta, tb); when
        // [ta - R, tb + R] lies inside [0, len], the edge covers the whole chord
        // of every such pixel's sphere (interior case, see walk_foot)
        interior = ta >= c.cull && tb <= len - c.cull;
        t_lo = fmaxf(ta, 0.0f);
        t_hi = fminf(tb, len);
    } else if (fabsf(az - zl) > c.cull) {
        return false;
    }
    if (t_lo > t_hi) return false;
    const float xa = fmaf(t_lo, ux, ax), xb = fmaf(t_hi, ux, ax);
    const float ya = fmaf(t_lo, uy, ay), yb = fmaf(t_hi, uy, ay);
    // pixel i has its centre at (i + 1/2) px
    const float fx0 = fmaf(fminf(xa, xb) - c.cull, c.inv_px, -0.5f);
    const float fx1 = fmaf(fmaxf(xa, xb) + c.cull, c.inv_px, -0.5f);
    const float fy0 = fmaf(fminf(ya, yb) - c.cull, c.inv_px, -0.5f);
    const float fy1 = fmaf(fmaxf(ya, yb) + c.cull, c.inv_px, -0.5f);
    const int i0 = max(0, (int)ceilf(fmaxf(fx0, -1.0f)));
    const int i1 = min(T - 1, (int)floorf(fminf(fx1, (float)T)));
    const int j0 = max(0, (int)ceilf(fmaxf(fy0, -1.0f)));
    const int j1 = min(T - 1, (int)floorf(fminf(fy1, (float)T)));
    if (i0 > i1 || j0 > j1) return false;
    const bool rows = fabsf(uy) >= fabsf(ux);
    const float au = rows ? ay : ax, av = rows ? ax : ay;
    const float uu = rows ? uy : ux, uv = rows ? ux : uy;
    const int u0 = rows ? j0 : i0, u1 = rows ? j1 : i1;
    const int v0 = rows ? i0 : j0, v1 = rows ? i1 : j1;
    const float a = fmaf(uu, uu, uz * uz);
    int W;
    if (a > 0.25f) {
        // approximate reciprocal and rsqrt: the span's 0.05-px margins absorb them
        const float inv_a = __fdividef(1.0f, a);
        const float hmax = c.cull * rsqrtf(a);
        const float base = fmaf(uv * inv_a, fmaf(fmaf(0.5f, c.fpx, -au), uu, (zl - az) * uz), av);
        f.c0 = fmaf(base - hmax, c.inv_px, -0.55f);
        f.c1 = uv * uu * inv_a;
        W = (int)floorf(fmaf(2.0f * hmax, c.inv_px, 0.101f)) + 1;
    } else {   // u = 0: a zero-length edge, its clipped box
        f.c0 = (float)v0;
        f.c1 = 0.0f;
        W = v1 - v0 + 1;
    }
    W = min(W, 255);
    const int weff = min(W, v1 - v0 + 1);
    const int n_rows = u1 - u0 + 1;
    const int passes = (n_rows * weff + 31) >> 5;
    f.w1 = (uint32_t)rec | ((uint32_t)interior << 14) | ((uint32_t)rows << 15) |
           ((uint32_t)W << 16) | ((uint32_t)passes << 24);
    f.geom = (uint32_t)u0 | ((uint32_t)n_rows << 8) | ((uint32_t)v0 << 16) | ((uint32_t)v1 << 24);
    return true;
}

template <int T>
constexpr int plane_pitch() {   // row pitch of a Sigma plane in shared memory (floats)
    return T + 8;
}

// The passes of one footprint: lane k of pass p takes index p * 32 + k of the
// dense range rows x span (row rr = index / weff, offset kk = index % weff,
// both exact in float for these small integers), evaluates the term at its
// pixel and adds w I to the layer's plane. Pixel coordinates relative to v_s
// are affine in the pixel indices: dx = i px + (px / 2 - a_x). INTERIOR: every
// pixel within R has its whole chord [t0 - w, t0 + w] on the edge, where the
// quartic's integral is (16/15) w^5 (the 3-point rule's value at m = 0, h = w).
template <int T, bool ROWS, bool INTERIOR, bool COUNT>
__device__ __forceinline__ void walk_foot(const Foot& fq, const float4 A, const float4 B,
                                          float zl, float* __restrict__ sig_l, const FpConst& c,
                                          int lane, uint32_t& n_nonzero, uint32_t& n_eval) {
    constexpr float P = (float)plane_pitch<T>();
    const float Wf = (float)((fq.w1 >> 16) & 0xffu);
    const int passes = (int)(fq.w1 >> 24);
    const float u0 = (float)(fq.geom & 0xffu);
    const float n_rows = (float)((fq.geom >> 8) & 0xffu);
    const float v0 = (float)((fq.geom >> 16) & 0xffu);
    const float v1 = (float)(fq.geom >> 24);
    const float weff = fminf(Wf, v1 - v0 + 1.0f);
    const float inv_w = __fdividef(1.0f, weff);   // floor((k + 1/2) / weff) is exact with it
    const float half_w = 0.5f * inv_w;
    const float ox = fmaf(0.5f, c.fpx, -A.x), oy = fmaf(0.5f, c.fpx, -A.y);
    const float dz = zl - A.z;
    const float dzuz = dz * B.y;
    const float wI = INTERIOR ? B.w * (16.0f / 15.0f) : B.w;
    for (int p = 0; p < passes; ++p) {
        const float idx = (float)(p * 32 + lane);
        const float rr = floorf(fmaf(idx, inv_w, half_w));
        const float kk = fmaf(-rr, weff, idx);
        const float u = u0 + rr;
        const float s = ceilf(fmaf(u, fq.c1, fq.c0));
        const float v = fmaxf(s, v0) + kk;
        const bool valid = rr < n_rows && v <= v1 && v < s + Wf;
        const float xi = ROWS ? v : u, yj = ROWS ? u : v;
        const float dx = fmaf(xi, c.fpx, ox), dy = fmaf(yj, c.fpx, oy);
        const float t0 = fmaf(dx, A.w, fmaf(dy, B.x, dzuz));
        const float ex = fmaf(-t0, A.w, dx);
        const float ey = fmaf(-t0, B.x, dy);
        const float ez = fmaf(-t0, B.y, dz);
        const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        const float h2 = fmaxf(c.R2 - d2, 0.0f);
        const float I = INTERIOR ? (h2 * h2) * sqrt_approx(h2) : segment_term_R4(t0, h2, B.z);
        if (valid) {
            float* q2 = sig_l + (int)fmaf(yj, P, xi);
            *q2 = fmaf(wI, I, *q2);
        }
        if (COUNT) {   // every lane of the pass is evaluated
            n_nonzero += valid && I > 0.0f;
            ++n_eval;
        }
    }
}

// One (tile, slab) of the field. Shared memory: S Sigma planes of T rows,
// then K staged records, then 32 footprints per warp.
template <int T, int S, bool COUNT>
__device__ __forceinline__ bool field_tile_fp(const csl_rec* __restrict__ recs,
                                              const uint32_t* __restrict__ tstart,
                                              const uint32_t* __restrict__ tend,
                                              const FpConst& c, float* __restrict__ sigma,
                                              uint32_t* __restrict__ mask,
                                              unsigned long long* __restrict__ n_pairs, int tile,
                                              int slab, unsigned char* smem, uint64_t* bar,
                                              uint32_t& phase) {
    constexpr int P = plane_pitch<T>();
    float* s_sig = reinterpret_cast<float*>(smem);
    float4* s_rec = reinterpret_cast<float4*>(smem + (size_t)S * T * P * sizeof(float));
    Foot* s_foot = reinterpret_cast<Foot*>(reinterpret_cast<unsigned char*>(s_rec) +
                                           (size_t)c.K * sizeof(csl_rec));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile % c.ntx, ty = tile / c.ntx;
    const uint32_t key = (uint32_t)slab * (uint32_t)c.n_tiles + (uint32_t)tile;
    const uint32_t beg = tstart[key], end = tend[key];
    const int l0 = slab * S;
    const int nl = min(S, c.n_layers - l0);
    const int l = warp;   // this warp's layer in the slab
    float* sig_l = s_sig + l * T * P;
    for (int q = lane; q < T * P / 4; q += 32)
        reinterpret_cast<float4*>(sig_l)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    Foot* my_foot = s_foot + warp * 32;
    uint32_t n_nonzero = 0, n_eval = 0;
    const float zl = (float)l * c.fdz;

    if (end > beg) {
        const float2 ox = c.org_x[tx], oy = c.org_y[ty], oz = c.org_z[slab];
        const float oxh = ox.x, oxl = ox.y, oyh = oy.x, oyl = oy.y, ozh = oz.x, ozl = oz.y;
        for (uint32_t c0 = beg; c0 < end; c0 += (uint32_t)c.K) {
            const int cnt = (int)min((uint32_t)c.K, end - c0);
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();   // the block's earlier reads of s_rec come first
                bulk_load(s_rec, recs + c0, (uint32_t)cnt * (uint32_t)sizeof(csl_rec), bar);
            }
            if (__syncthreads_or(!mbar_wait(bar, phase))) {
                if (threadIdx.x == 0) atomicOr(c.err, ST_TIMEOUT);
                mbar_wait(bar, phase);
                return false;
            }
            phase ^= 1u;
            for (int r = threadIdx.x; r < cnt; r += 32 * S) {
                const float4 r0 = s_rec[2 * r], r1 = s_rec[2 * r + 1];
                s_rec[2 * r] =
                    make_float4((r0.x - oxh) - oxl, (r0.y - oyh) - oyl, (r0.z - ozh) - ozl, r0.w);
                s_rec[2 * r + 1] = make_float4(r1.x, r1.y, r1.z, r1.w * c.inv_R4);
            }
            __syncthreads();
            if (l < nl) {
                for (int r0 = 0; r0 < cnt; r0 += 32) {
                    const int r = r0 + lane;
                    Foot f;
                    const bool ok = r < cnt && make_foot<T>(s_rec[2 * r], s_rec[2 * r + 1], zl, r,
                                                            c, f);
                    const uint32_t ball = __ballot_sync(0xffffffffu, ok);
                    if (ok) my_foot[__popc(ball & ((1u << lane) - 1u))] = f;
                    __syncwarp();
                    const int n = __popc(ball);
                    for (int q = 0; q < n; ++q) {
                        const Foot fq = my_foot[q];
                        const int rec = (int)(fq.w1 & 0x3fffu);
                        const float4 A = s_rec[2 * rec], B = s_rec[2 * rec + 1];
                        switch ((fq.w1 >> 14) & 3u) {   // interior | rows << 1, warp-uniform
                            case 0: walk_foot<T, false, false, COUNT>(fq, A, B, zl, sig_l, c, lane, n_nonzero, n_eval); break;
                            case 1: walk_foot<T, false, true, COUNT>(fq, A, B, zl, sig_l, c, lane, n_nonzero, n_eval); break;
                            case 2: walk_foot<T, true, false, COUNT>(fq, A, B, zl, sig_l, c, lane, n_nonzero, n_eval); break;
                            default: walk_foot<T, true, true, COUNT>(fq, A, B, zl, sig_l, c, lane, n_nonzero, n_eval); break;
                        }
                    }
                    __syncwarp();   // the next group overwrites the footprints
                }
            }
            __syncthreads();   // the next chunk reuses s_rec
        }
    }
    if (COUNT) {   // n_pairs[0]: nonzero terms, n_pairs[1]: evaluated terms
        unsigned long long t = n_nonzero, e = n_eval;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_down_sync(0xffffffffu, t, o);
            e += __shfl_down_sync(0xffffffffu, e, o);
        }
        if (lane == 0 && t) atomicAdd(n_pairs, t);
        if (lane == 0 && e) atomicAdd(n_pairs + 1, e);
    }
    __syncwarp();
    if (l >= nl) return true;
    const int gx = tx * T, gy = ty * T;
    const int wx = min(T, c.nx - gx), wy = min(T, c.ny - gy);
    float* dst = sigma ? sigma + (int64_t)(l0 + l) * c.ny * c.nx : nullptr;
    // Sigma plane and inside mask of this warp's layer; rows of 32 / T pixels per step
    constexpr int RPS = 32 / T;   // rows per step
    const int col = lane % T, sub = lane / T;
    uint32_t my_bits = 0;
    for (int j0 = 0; j0 < T; j0 += RPS) {
        const int j = j0 + sub;
        const float v = sig_l[j * P + col];
        const bool in = col < wx && j < wy;
        if (dst && in) dst[(int64_t)(gy + j) * c.nx + gx + col] = v;
        const uint32_t b = __ballot_sync(0xffffffffu, in && v >= c.C);
        if (lane == j0 / RPS) my_bits = b;
    }
    if (mask && lane < T / RPS) {
        // row group `lane`: RPS rows of T bits each; pixel i is padded sample i + 1
        const int I0 = gx + 1;
        const int sh = I0 & 31;
#pragma unroll
        for (int k = 0; k < RPS; ++k) {
            constexpr uint32_t kRowBits = T == 32 ? 0xffffffffu : ((1u << (T & 31)) - 1u);
            const uint32_t bits = (my_bits >> ((k * T) & 31)) & kRowBits;
            if (!bits) continue;
            const int J = gy + lane * RPS + k + 1;
            uint32_t* row = mask + (int64_t)(l0 + l) * c.mask_wpl + (int64_t)J * c.mwr;
            atomicOr(row + (I0 >> 5), bits << sh);
            const uint32_t hi = sh ? bits >> (32 - sh) : 0u;
            if (hi) atomicOr(row + (I0 >> 5) + 1, hi);
        }
    }
    return true;
}

template <int T, int S, bool COUNT>
__global__ void __launch_bounds__(32 * S)
k_field_fp(const csl_rec* __restrict__ recs, const uint32_t* __restrict__ tstart,
           const uint32_t* __restrict__ tend, FpConst c, float* __restrict__ sigma,
           uint32_t* __restrict__ mask, unsigned long long* __restrict__ n_pairs) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    field_tile_fp<T, S, COUNT>(recs, tstart, tend, c, sigma, mask, n_pairs, blockIdx.x,
                               blockIdx.y, smem, &bar, phase);
}

template <int T, int S>
size_t fp_smem_bytes(int K) {
    return (size_t)S * T * plane_pitch<T>() * sizeof(float) + (size_t)K * sizeof(csl_rec) +
           (size_t)S * 32 * sizeof(Foot);
}

template <int T, int S, bool COUNT>
void launch_fp(const FpConst& c, dim3 grid, const csl_rec* recs, const uint32_t* ts,
               const uint32_t* te, float* sigma, uint32_t* mask, unsigned long long* count,
               cudaStream_t s) {
    const size_t smem = fp_smem_bytes<T, S>(c.K);
    auto kern = k_field_fp<T, S, COUNT>;
    CSL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 32 * S, smem, s>>>(recs, ts, te, c, sigma, mask, count);
}

template <int T, int S>
void launch_fp_count(const FpConst& c, dim3 grid, const csl_rec* recs, const uint32_t* ts,
                     const uint32_t* te, float* sigma, uint32_t* mask, unsigned long long* count,
                     cudaStream_t s) {
    if (count) launch_fp<T, S, true>(c, grid, recs, ts, te, sigma, mask, count, s);
    else launch_fp<T, S, false>(c, grid, recs, ts, te, sigma, mask, nullptr, s);
}

}  // namespace

void field_chunk_fp(const ChunkGeom& g, const SlabBins& bins, float C, const float2* org,
                    uint32_t* err, float* sigma, uint32_t* mask, unsigned long long* count_pairs,
                    cudaStream_t s) {
    FpConst c;
    c.nx = g.nx;
    c.ny = g.ny;
    c.ntx = g.ntx;
    c.n_tiles = g.ntx * g.nty;
    c.n_layers = g.n_layers;
    c.K = g.K;
    c.R2 = (float)(g.R * g.R);
    c.inv_R4 = (float)(1.0 / (g.R * g.R * g.R * g.R));
    c.fpx = (float)g.px;
    c.inv_px = (float)(1.0 / g.px);
    c.fdz = (float)g.dz;
    c.cull = (float)(g.R * (1.0 + 1e-5) + 1e-6);
    c.C = C;
    c.org_x = org;
    c.org_y = org + g.ntx;
    c.org_z = org + g.ntx + g.nty;
    c.mwr = (int32_t)mask_words_per_row(g.nx);
    c.mask_wpl = mask_words_per_layer(g.nx, g.ny);
    c.err = err;
    if (c.K < 32 || c.K > 1024 || c.K % 32) fail(CSL_ERR_INVALID_ARG, "staging chunk K");
    dim3 grid((unsigned)c.n_tiles, (unsigned)g.n_slabs);
    const csl_rec* recs = bins.recs.as<csl_rec>();
    const uint32_t* ts = bins.tile_start.as<uint32_t>();
    const uint32_t* te = bins.tile_end.as<uint32_t>();
#define CSL_FP_CASE(TV, SV)                                                                \
    if (g.T == TV && g.S == SV) {                                                          \
        launch_fp_count<TV, SV>(c, grid, recs, ts, te, sigma, mask, count_pairs, s);       \
        CSL_LAUNCH_CHECK("footprint field");                                               \
        return;                                                                            \
    }
    CSL_FP_CASE(16, 1)
    CSL_FP_CASE(16, 2)
    CSL_FP_CASE(16, 4)
    CSL_FP_CASE(16, 8)
    CSL_FP_CASE(32, 1)
    CSL_FP_CASE(32, 2)
    CSL_FP_CASE(32, 4)
    CSL_FP_CASE(32, 8)
#undef CSL_FP_CASE
    fail(CSL_ERR_INVALID_ARG, "footprint field: tile 16 or 32, slab 1, 2, 4 or 8");
}

}  // namespace csl
