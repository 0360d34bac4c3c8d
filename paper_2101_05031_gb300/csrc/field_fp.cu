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

#include <string.h>

#include <algorithm>
#include <vector>

#include "field_tile.cuh"
#include "slice.cuh"

namespace csl {
namespace {

struct FpConst {
    int32_t nx, ny, ntx, nty, n_tiles;
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
    // fused pass (FusedVerts): tables, vertices, saddle bits, allocation counter
    uint32_t* tbase;
    uint16_t* roff;
    float2* verts;
    uint32_t* saddle;
    uint32_t* counter;
    uint32_t cap;
    float fx0, fy0;      // grid origin as the contour stage takes it (float)
};

// One (record, layer) footprint with the constants its walk uses, built by
// one lane per record (so the set-up is paid once per 16 records and layer
// rather than once per footprint by the whole warp), 80 bytes: the span of
// row (or column) u starts at ceil(c0 + u c1) and is W pixels wide, clipped to
// [v0, v1]; weff = min(W, v1 - v0 + 1); inv_w = 1 / weff (approximate: the
// row index floor((k + 1/2) inv_w) is exact with it for these small
// integers); pixel coordinates relative to v_s are dx = i px + ox, dy = j px
// + oy, dz (and dz u_z); wI = w / R^4 (times 16/15 for the interior closed
// form); bits = record (< 2^14) | interior << 14 | mode << 15.
struct __align__(16) Foot {
    float inv_w, weff, u0, n_rows;
    float c0, c1, v0, v1;
    float Wf, ox, oy, dz;
    float dzuz, wI, ux, uy;
    float uz, len;
    uint32_t bits, passes;
};
static_assert(sizeof(Foot) == 80, "Foot is five 16-byte words");

// records per footprint-building round (one lane each); the warp's queue holds
// one round's footprints
constexpr int kFootGroup = 16;

// Footprint of record (A, B) in layer plane zl of a T x T tile; false when
// the edge's support misses the tile in that plane.
template <int T, int EXT>
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
    // tile-local pixels 0 .. EXT (EXT = T - 1, or T with the fused pass's halo)
    const int i0 = max(0, (int)ceilf(fmaxf(fx0, -1.0f)));
    const int i1 = min(EXT, (int)floorf(fminf(fx1, (float)(EXT + 1))));
    const int j0 = max(0, (int)ceilf(fmaxf(fy0, -1.0f)));
    const int j1 = min(EXT, (int)floorf(fminf(fy1, (float)(EXT + 1))));
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
    const int weff = min(W, v1 - v0 + 1);
    const int n_rows = u1 - u0 + 1;
    f.weff = (float)weff;
    f.inv_w = __fdividef(1.0f, f.weff);
    f.u0 = (float)u0;
    f.n_rows = (float)n_rows;
    f.v0 = (float)v0;
    f.v1 = (float)v1;
    f.Wf = (float)W;
    f.ox = fmaf(0.5f, c.fpx, -ax);
    f.oy = fmaf(0.5f, c.fpx, -ay);
    f.dz = zl - az;
    f.dzuz = f.dz * uz;
    f.wI = interior ? B.w * (16.0f / 15.0f) : B.w;
    f.ux = ux;
    f.uy = uy;
    f.uz = uz;
    f.len = len;
    f.bits = (uint32_t)rec | ((uint32_t)interior << 14) | ((uint32_t)rows << 15);
    f.passes = (uint32_t)((n_rows * weff + 31) >> 5);
    return true;
}

// Row pitch of a Sigma plane in shared memory (floats): T + 1 puts the rows of
// a column-mode footprint in distinct banks; the fused pass's planes have T + 1
// rows, so its pitch keeps the planes 16-byte multiples.
template <int T, bool FUSED>
constexpr int plane_pitch() {
    return FUSED ? T + 8 : T + 1;
}

// The passes of one footprint: lane k of pass p takes index p * 32 + k of the
// dense range rows x span (row rr = index / weff, offset kk = index % weff,
// both exact in float for these small integers), evaluates the term at its
// pixel and adds w I to the layer's plane. Pixel coordinates relative to v_s
// are affine in the pixel indices: dx = i px + (px / 2 - a_x). INTERIOR: every
// pixel within R has its whole chord [t0 - w, t0 + w] on the edge, where the
// quartic's integral is (16/15) w^5 (the 3-point rule's value at m = 0, h = w).
template <int T, bool ROWS, bool INTERIOR, bool COUNT, bool FUSED>
__device__ __forceinline__ void walk_foot(const Foot& fq, const float2 An,
                                          float* __restrict__ sig_l, const FpConst& c, int lane,
                                          uint32_t& n_nonzero, uint32_t& n_eval) {
    constexpr float P = (float)plane_pitch<T, FUSED>();
    const float half_w = 0.5f * fq.inv_w;
    // the fused pass's halo (column T, row T) in the next tiles' frames (An: v_s
    // relative to their corners), so that its values are the ones those tiles
    // compute for their first column and row, bit for bit
    const float oxn = FUSED ? fmaf(0.5f, c.fpx, -An.x) : 0.0f;
    const float oyn = FUSED ? fmaf(0.5f, c.fpx, -An.y) : 0.0f;
    float idx = (float)lane;
    for (uint32_t p = 0; p < fq.passes; ++p, idx += 32.0f) {
        const float rr = floorf(fmaf(idx, fq.inv_w, half_w));
        const float kk = fmaf(-rr, fq.weff, idx);
        const float u = fq.u0 + rr;
        const float s = ceilf(fmaf(u, fq.c1, fq.c0));
        const float v = fmaxf(s, fq.v0) + kk;
        const bool valid = rr < fq.n_rows && v <= fq.v1 && v < s + fq.Wf;
        const float xi = ROWS ? v : u, yj = ROWS ? u : v;
        float dx = fmaf(xi, c.fpx, fq.ox), dy = fmaf(yj, c.fpx, fq.oy);
        if (FUSED) {
            if (xi == (float)T) dx = fmaf(0.0f, c.fpx, oxn);
            if (yj == (float)T) dy = fmaf(0.0f, c.fpx, oyn);
        }
        const float t0 = fmaf(dx, fq.ux, fmaf(dy, fq.uy, fq.dzuz));
        const float ex = fmaf(-t0, fq.ux, dx);
        const float ey = fmaf(-t0, fq.uy, dy);
        const float ez = fmaf(-t0, fq.uz, fq.dz);
        const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        const float h2 = fmaxf(c.R2 - d2, 0.0f);
        const float I = INTERIOR ? (h2 * h2) * sqrt_approx(h2) : segment_term_R4(t0, h2, fq.len);
        if (valid) {
            float* q2 = sig_l + (int)fmaf(yj, P, xi);
            *q2 = fmaf(fq.wI, I, *q2);
        }
        if (COUNT) {   // every lane of the pass is evaluated
            n_nonzero += valid && I > 0.0f;
            ++n_eval;
        }
    }
}

// The fused pass's contour inputs of one layer (warp): the tile's crossing
// vertices in edge-id order, their row offsets and list base, and the
// saddle-join bits (FusedVerts). sig_l holds Sigma of the tile's pixels and of
// its next column and row (those computed in the next tiles' frames, so equal
// to what they compute); pixels outside the grid count as 0 (outside), like
// the padding ring. Each row's inside samples are one 64-bit word, bit a + 1
// for tile-local column a in [-1, T] (column -1: the padding sample before the
// first tile column, always outside); the crossing bits of a row are then
// in ^ (in >> 1) (x edges) and in ^ (the row above) (y edges), as the contour
// stage derives them from the mask. Vertex and saddle expressions are the
// contour stage's.
template <int T>
__device__ __forceinline__ void fused_epilogue(const float* __restrict__ sig_l, const FpConst& c,
                                               int tx, int ty, int tile, int64_t lg, int lane,
                                               unsigned char* scratch) {
    constexpr int P = plane_pitch<T, true>();
    uint64_t* s_in = reinterpret_cast<uint64_t*>(scratch);           // rows -1 .. T
    uint16_t* s_roff = reinterpret_cast<uint16_t*>(scratch + (T + 2) * 8);
    const int gx = tx * T, gy = ty * T;
    auto val = [&](int a, int b) -> float {
        return (a >= 0 && b >= 0 && a <= T && b <= T && gx + a < c.nx && gy + b < c.ny)
                   ? sig_l[b * P + a]
                   : 0.0f;
    };
    // inside words of rows -1 .. T
    for (int b = -1; b <= T; ++b) {
        const bool in_l = lane <= T && val(lane, b) >= c.C;          // columns 0 .. 31 (T = 16: .. 16)
        const uint32_t bl = __ballot_sync(0xffffffffu, in_l);
        const bool in_t = T == 32 && val(T, b) >= c.C;                // column 32 (T = 32 only)
        if (lane == 0) s_in[b + 1] = ((uint64_t)bl << 1) | ((uint64_t)in_t << (T + 1));
    }
    __syncwarp();
    const int a_hi = min(T - 1, c.nx - 1 - gx), b_hi = min(T - 1, c.ny - 1 - gy);
    const int a_lo = tx == 0 ? -1 : 0, b_lo = ty == 0 ? -1 : 0;
    // owned samples: bits a_lo + 1 .. a_hi + 1
    const uint64_t own = ((2ull << (a_hi + 1)) - 1ull) & ~((1ull << (a_lo + 1)) - 1ull);
    uint32_t total = 0;
    for (int b = -1; b < T; ++b) {
        uint32_t cnt = 0;
        if (b >= b_lo && b <= b_hi) {
            const uint64_t in = s_in[b + 1], up = s_in[b + 2];
            cnt = __popcll((in ^ (in >> 1)) & own) + __popcll((in ^ up) & own);
        }
        if (lane == 0) s_roff[b + 1] = (uint16_t)total;
        total += cnt;
    }
    __syncwarp();
    const int64_t tl = lg * c.n_tiles + tile;
    for (int k = lane; k <= T; k += 32) c.roff[tl * (T + 1) + k] = s_roff[k];
    uint32_t base = 0;
    if (lane == 0) {
        base = atomicAdd(c.counter, total);
        if ((uint64_t)base + total > c.cap) atomicOr(c.counter + 1, 1u);
        c.tbase[tl] = base;
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((uint64_t)base + total > c.cap) return;   // reported: the chunk runs again
    for (int b = b_lo; b <= b_hi; ++b) {
        const uint64_t in = s_in[b + 1], up = s_in[b + 2];
        const uint64_t hx = (in ^ (in >> 1)) & own, vy = (in ^ up) & own;
        const int J = gy + b + 1;
        const uint32_t row0 = base + s_roff[b + 1];
        // column -1 (first tile column): its x edge from the padding sample to pixel 0
        if ((hx & 1ull) && lane == 0) {
            const float sa = val(0, b);
            const float t = __fdividef(sa - c.C, sa - 0.0f);
            const float xp = 0.0f + 0.5f - t;
            c.verts[row0] = make_float2(c.fx0 + xp * c.fpx, c.fy0 + ((float)J - 0.5f) * c.fpx);
        }
        // columns 0 .. T - 1: lane a, bit a + 1
        const int a = lane;
        const int q = a + 1;
        const bool hb = q <= T && ((hx >> q) & 1ull);
        const bool vb = q <= T && ((vy >> q) & 1ull);
        if (hb || vb) {
            const uint64_t below = (1ull << q) - 1ull;
            const uint32_t pos = row0 + __popcll(hx & below) + __popcll(vy & below);
            const int I = gx + a + 1;
            const float v0 = val(a, b);
            const bool in0 = v0 >= c.C;
            if (hb) {   // x edge (I, J) -> (I + 1, J)
                const float v1 = val(a + 1, b);
                const float sa = in0 ? v0 : v1, sbv = in0 ? v1 : v0;
                const float t = __fdividef(sa - c.C, sa - sbv);
                const float xp = in0 ? ((float)I - 0.5f + t) : ((float)I + 0.5f - t);
                c.verts[pos] = make_float2(c.fx0 + xp * c.fpx, c.fy0 + ((float)J - 0.5f) * c.fpx);
            }
            if (vb) {   // y edge (I, J) -> (I, J + 1)
                const float v3 = val(a, b + 1);
                const float sa = in0 ? v0 : v3, sbv = in0 ? v3 : v0;
                const float t = __fdividef(sa - c.C, sa - sbv);
                const float yp = in0 ? ((float)J - 0.5f + t) : ((float)J + 0.5f - t);
                c.verts[pos + (hb ? 1u : 0u)] =
                    make_float2(c.fx0 + ((float)I - 0.5f) * c.fpx, c.fy0 + yp * c.fpx);
            }
        }
        // saddle cells (a, b), a, b >= 0: inside corners on one diagonal only
        if (b >= 0) {
            const uint64_t c0 = in, c1 = in >> 1, c3 = up, c2 = up >> 1;
            const uint64_t sad = ((c0 & c2 & ~c1 & ~c3) | (c1 & c3 & ~c0 & ~c2)) & own & ~1ull;
            if (sad) {
                bool joined = false;
                if (q <= T && ((sad >> q) & 1ull)) {
                    const float w0 = val(a, b), w1 = val(a + 1, b), w2 = val(a + 1, b + 1),
                                w3 = val(a, b + 1);
                    joined = 0.25f * (w0 + w1 + w2 + w3) >= c.C;
                }
                const uint32_t sb = __ballot_sync(0xffffffffu, joined);
                if (lane == 0 && sb) {
                    uint32_t* row = c.saddle + lg * c.mask_wpl + (int64_t)J * c.mwr;
                    const int sh = (gx + 1) & 31;
                    atomicOr(row + ((gx + 1) >> 5), sb << sh);
                    const uint32_t hi = sh ? sb >> (32 - sh) : 0u;
                    if (hi) atomicOr(row + ((gx + 1) >> 5) + 1, hi);
                }
            }
        }
    }
}

// One (tile, slab) of the field. Shared memory: S Sigma planes of T rows,
// then K staged records, then kFootGroup footprints per warp.
template <int T, int S, bool COUNT, bool FUSED>
__device__ __forceinline__ bool field_tile_fp(const csl_rec* __restrict__ recs,
                                              const uint32_t* __restrict__ tstart,
                                              const uint32_t* __restrict__ tend,
                                              const FpConst& c, float* __restrict__ sigma,
                                              uint32_t* __restrict__ mask,
                                              unsigned long long* __restrict__ n_pairs, int tile,
                                              int slab, unsigned char* smem, uint64_t* bar,
                                              uint32_t& phase) {
    constexpr int P = plane_pitch<T, FUSED>();
    constexpr int ROWS = FUSED ? T + 1 : T;   // the fused pass also evaluates the next row
    float* s_sig = reinterpret_cast<float*>(smem);
    float4* s_rec = reinterpret_cast<float4*>(smem + (size_t)S * ROWS * P * sizeof(float));
    // the fused pass keeps each record's v_s.xy also relative to the next tiles' corners
    float2* s_recn = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(s_rec) +
                                               (size_t)c.K * sizeof(csl_rec));
    Foot* s_foot = reinterpret_cast<Foot*>(reinterpret_cast<unsigned char*>(s_recn) +
                                           (FUSED ? (size_t)c.K * sizeof(float2) : 0));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile % c.ntx, ty = tile / c.ntx;
    const uint32_t key = (uint32_t)slab * (uint32_t)c.n_tiles + (uint32_t)tile;
    const uint32_t beg = tstart[key], end = tend[key];
    const int l0 = slab * S;
    const int nl = min(S, c.n_layers - l0);
    const int l = warp;   // this warp's layer in the slab
    float* sig_l = s_sig + l * ROWS * P;
    for (int q = lane; q < ROWS * P / 4; q += 32)
        reinterpret_cast<float4*>(sig_l)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    Foot* my_foot = s_foot + warp * kFootGroup;
    uint32_t n_nonzero = 0, n_eval = 0;
    const float zl = (float)l * c.fdz;

    if (end > beg) {
        const float2 ox = c.org_x[tx], oy = c.org_y[ty], oz = c.org_z[slab];
        const float oxh = ox.x, oxl = ox.y, oyh = oy.x, oyl = oy.y, ozh = oz.x, ozl = oz.y;
        // the next tile column's and row's corners (the fused pass's halo); past
        // the grid's last tile the halo lies outside and its values are not used
        const float2 oxn = FUSED ? c.org_x[min(tx + 1, c.ntx - 1)] : ox;
        const float2 oyn = FUSED ? c.org_y[min(ty + 1, c.nty - 1)] : oy;
        const float oxnh = oxn.x, oxnl = oxn.y, oynh = oyn.x, oynl = oyn.y;
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
                if (FUSED)
                    s_recn[r] = make_float2((r0.x - oxnh) - oxnl, (r0.y - oynh) - oynl);
                s_rec[2 * r] =
                    make_float4((r0.x - oxh) - oxl, (r0.y - oyh) - oyl, (r0.z - ozh) - ozl, r0.w);
                s_rec[2 * r + 1] = make_float4(r1.x, r1.y, r1.z, r1.w * c.inv_R4);
            }
            __syncthreads();
            if (l < nl) {
                for (int r0 = 0; r0 < cnt; r0 += kFootGroup) {
                    const int r = r0 + lane;
                    Foot f;
                    const bool ok = lane < kFootGroup && r < cnt &&
                                    make_foot<T, FUSED ? T : T - 1>(s_rec[2 * r], s_rec[2 * r + 1],
                                                                    zl, r, c, f);
                    const uint32_t ball = __ballot_sync(0xffffffffu, ok);
                    if (ok) my_foot[__popc(ball & ((1u << lane) - 1u))] = f;
                    __syncwarp();
                    const int n = __popc(ball);
                    for (int q = 0; q < n; ++q) {
                        const Foot fq = my_foot[q];
                        const float2 An =
                            FUSED ? s_recn[fq.bits & 0x3fffu] : make_float2(0.0f, 0.0f);
                        switch ((fq.bits >> 14) & 3u) {   // interior | rows << 1, warp-uniform
                            case 0: walk_foot<T, false, false, COUNT, FUSED>(fq, An, sig_l, c, lane, n_nonzero, n_eval); break;
                            case 1: walk_foot<T, false, true, COUNT, FUSED>(fq, An, sig_l, c, lane, n_nonzero, n_eval); break;
                            case 2: walk_foot<T, true, false, COUNT, FUSED>(fq, An, sig_l, c, lane, n_nonzero, n_eval); break;
                            default: walk_foot<T, true, true, COUNT, FUSED>(fq, An, sig_l, c, lane, n_nonzero, n_eval); break;
                        }
                    }
                    __syncwarp();   // the next group overwrites the footprints
                }
            }
            // the next chunk reuses s_rec; after the last one each warp goes on to
            // its own plane (no other warp's data) without waiting
            if (c0 + (uint32_t)c.K < end) __syncthreads();
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
    if (FUSED)
        fused_epilogue<T>(sig_l, c, tx, ty, tile, (int64_t)(l0 + l), lane,
                          reinterpret_cast<unsigned char*>(my_foot));
    return true;
}

template <int T, int S, bool COUNT, bool FUSED>
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
    field_tile_fp<T, S, COUNT, FUSED>(recs, tstart, tend, c, sigma, mask, n_pairs, blockIdx.x,
                                      blockIdx.y, smem, &bar, phase);
}

// One job of a batch for the persistent footprint kernel.
struct FpJob {
    FpConst c;
    const csl_rec* recs;   // the binned records, in list order
    const uint32_t* tstart;
    const uint32_t* tend;
    float* sigma;
    uint32_t* mask;
};
static_assert(sizeof(FpJob) % 4 == 0, "FpJob is copied as 32-bit words");

// Persistent footprint field kernel over the (job, slab, tile) items of a
// batch, in the order `order` gives (longest tile lists first): each CTA takes
// the next item from a shared counter. Every job has the same tile side, slab
// depth and staging chunk.
template <int T, int S>
__global__ void __launch_bounds__(32 * S)
k_field_fp_batch(const FpJob* __restrict__ jobs, const uint2* __restrict__ items,
                 const uint32_t* __restrict__ order, uint32_t n_items, uint32_t* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ FpJob s_job;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    uint32_t cur_job = 0xffffffffu;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const uint2 item = items[order[it]];
        if (item.x != cur_job) {   // consecutive items often belong to the same job
            cur_job = item.x;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(jobs + item.x);
            for (int i = threadIdx.x; i < (int)(sizeof(FpJob) / 4); i += 32 * S)
                reinterpret_cast<uint32_t*>(&s_job)[i] = src[i];
            __syncthreads();
        }
        const uint32_t n_tiles = (uint32_t)s_job.c.n_tiles;
        if (!field_tile_fp<T, S, false, false>(s_job.recs, s_job.tstart, s_job.tend, s_job.c,
                                               s_job.sigma, s_job.mask, nullptr,
                                               (int)(item.y % n_tiles), (int)(item.y / n_tiles),
                                               smem, &bar, phase))
            break;   // a bulk copy gave up (reported): this CTA takes no more items
        __syncthreads();   // shared memory is reused by the next item
    }
}

template <int T, int S, bool FUSED>
size_t fp_smem_bytes(int K) {
    return (size_t)S * (FUSED ? T + 1 : T) * plane_pitch<T, FUSED>() * sizeof(float) +
           (size_t)K * sizeof(csl_rec) + (FUSED ? (size_t)K * sizeof(float2) : 0) +
           (size_t)S * kFootGroup * sizeof(Foot);
}

template <int T, int S, bool COUNT, bool FUSED>
void launch_fp(const FpConst& c, dim3 grid, const csl_rec* recs, const uint32_t* ts,
               const uint32_t* te, float* sigma, uint32_t* mask, unsigned long long* count,
               cudaStream_t s) {
    const size_t smem = fp_smem_bytes<T, S, FUSED>(c.K);
    auto kern = k_field_fp<T, S, COUNT, FUSED>;
    CSL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 32 * S, smem, s>>>(recs, ts, te, c, sigma, mask, count);
}

template <int T, int S>
void launch_fp_count(const FpConst& c, dim3 grid, const csl_rec* recs, const uint32_t* ts,
                     const uint32_t* te, float* sigma, uint32_t* mask, unsigned long long* count,
                     cudaStream_t s, bool fused) {
    if (fused) {
        if (count) launch_fp<T, S, true, true>(c, grid, recs, ts, te, sigma, mask, count, s);
        else launch_fp<T, S, false, true>(c, grid, recs, ts, te, sigma, mask, nullptr, s);
    } else {
        if (count) launch_fp<T, S, true, false>(c, grid, recs, ts, te, sigma, mask, count, s);
        else launch_fp<T, S, false, false>(c, grid, recs, ts, te, sigma, mask, nullptr, s);
    }
}


FpConst make_fp_const(const ChunkGeom& g, float C, const float2* org, uint32_t* err) {
    FpConst c{};
    c.nx = g.nx;
    c.ny = g.ny;
    c.ntx = g.ntx;
    c.nty = g.nty;
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
    c.fx0 = (float)g.x0;
    c.fy0 = (float)g.y0;
    return c;
}

}  // namespace

void field_chunk_fp(const ChunkGeom& g, const SlabBins& bins, float C, const float2* org,
                    uint32_t* err, float* sigma, uint32_t* mask, unsigned long long* count_pairs,
                    cudaStream_t s, FusedVerts* fv) {
    FpConst c = make_fp_const(g, C, org, err);
    const bool fused = g.fused;
    if (fused != (fv != nullptr) || (fused && !mask))
        fail(CSL_ERR_INVALID_ARG, "fused pass: vertex lists and mask are required");
    c.tbase = fused ? fv->tbase.as<uint32_t>() : nullptr;
    c.roff = fused ? fv->roff.as<uint16_t>() : nullptr;
    c.verts = fused ? fv->verts.as<float2>() : nullptr;
    c.saddle = fused ? fv->saddle.as<uint32_t>() : nullptr;
    c.counter = fused ? fv->counter.as<uint32_t>() : nullptr;
    c.cap = fused ? (uint32_t)std::min<int64_t>(fv->cap, 0xffffffffLL) : 0u;
    if (c.K < 32 || c.K > 1024 || c.K % 32) fail(CSL_ERR_INVALID_ARG, "staging chunk K");
    dim3 grid((unsigned)c.n_tiles, (unsigned)g.n_slabs);
    const csl_rec* recs = bins.recs.as<csl_rec>();
    const uint32_t* ts = bins.tile_start.as<uint32_t>();
    const uint32_t* te = bins.tile_end.as<uint32_t>();
#define CSL_FP_CASE(TV, SV)                                                                \
    if (g.T == TV && g.S == SV) {                                                          \
        launch_fp_count<TV, SV>(c, grid, recs, ts, te, sigma, mask, count_pairs, s, fused); \
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

// Batch jobs for the persistent footprint kernel (device array of FpJob).
void fp_batch_jobs(const std::vector<FieldBatchJob>& jobs, const float2* const* orgs,
                   std::vector<unsigned char>& host) {
    host.assign(jobs.size() * sizeof(FpJob), 0);
    for (size_t j = 0; j < jobs.size(); ++j) {
        const FieldBatchJob& J = jobs[j];
        FpJob f;
        f.c = make_fp_const(J.g, (float)J.L->C, orgs[j], J.err);
        f.recs = J.bins->recs.as<csl_rec>();
        f.tstart = J.bins->tile_start.as<uint32_t>();
        f.tend = J.bins->tile_end.as<uint32_t>();
        f.sigma = J.sigma;
        f.mask = J.mask;
        memcpy(host.data() + j * sizeof(FpJob), &f, sizeof(FpJob));
    }
}

void fp_batch_launch(const void* jobs, const uint2* items, const uint32_t* order, uint32_t n,
                     uint32_t* counter, int T, int S, int K, int n_ctas, cudaStream_t s) {
    const FpJob* J = static_cast<const FpJob*>(jobs);
#define CSL_FPB_CASE(TV, SV)                                                                 \
    if (T == TV && S == SV) {                                                                \
        const size_t smem = fp_smem_bytes<TV, SV, false>(K);                                 \
        CSL_CUDA(cudaFuncSetAttribute(k_field_fp_batch<TV, SV>,                              \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_field_fp_batch<TV, SV><<<n_ctas, 32 * SV, smem, s>>>(J, items, order, n, counter);  \
        CSL_LAUNCH_CHECK("batch footprint field");                                           \
        return;                                                                              \
    }
    CSL_FPB_CASE(16, 2)
    CSL_FPB_CASE(16, 4)
    CSL_FPB_CASE(16, 8)
    CSL_FPB_CASE(32, 2)
    CSL_FPB_CASE(32, 4)
    CSL_FPB_CASE(32, 8)
#undef CSL_FPB_CASE
    fail(CSL_ERR_INVALID_ARG, "batch footprint field: tile 16 or 32, slab 2, 4 or 8");
}

}  // namespace csl
