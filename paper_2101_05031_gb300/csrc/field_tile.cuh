// Device helpers shared by the field kernel and the volume-fraction adjoint:
// staging one edge record for a (16x16-pixel tile, slab) CTA, the per-warp
// cull mask, and the closed-form segment integral (Eq. 7) by 3-point
// Gauss-Legendre on the clipped interval.
#pragma once

#include "lattice.cuh"

namespace csl {

constexpr int kTileWarps = 8;   // a CTA = 8 warps, each an 8 x 4 pixel block

struct TileCull {
    float fpx, fdz;      // pixel size, layer spacing (float)
    float cull;          // R plus rounding slack
    float cull_line2;    // (cull + half-diagonal of a warp's pixel block)^2
    float inv_R4;
};

// ---- bulk copy (TMA) into shared memory, completion on an mbarrier ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
// makes the initialised barrier visible to the asynchronous (bulk copy) proxy
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's (and, after a barrier, the block's) ordinary shared
// memory accesses before the bulk copy's writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one arrival that also expects `bytes` of transactions, then the copy of
// `bytes` (a multiple of 16, both addresses 16-byte aligned) from global memory
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}
// Waits for the barrier's phase `parity` to complete, at most kWaitLimit polls
// (each may suspend the thread for a while); false when it gave up.
constexpr uint32_t kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Loads record rp, converts it to coordinates relative to the tile corner and
// the slab's first layer plane (each given as a (hi, lo) float pair) and
// returns its cull mask: bit w * 8 + l is set when the edge's support (radius
// cull) may reach a pixel centre of warp w's 8 x 4 block at layer l < nl,
// i.e. when the block meets the xy box of the edge clipped to |z - z_l| <= cull
// grown by cull, and the block's centre lies within cull + half-diagonal of
// the edge's line. A = (ax, ay, az, ux), B = (uy, uz, len, w / R^4).
__device__ __forceinline__ uint64_t stage_record(const csl_rec* rp_rec, float oxh, float oxl,
                                                 float oyh, float oyl, float ozh, float ozl, int nl,
                                                 const TileCull& c, float4& A, float4& B) {
    const float4* rp = reinterpret_cast<const float4*>(rp_rec);
    const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
    const float ax = (r0.x - oxh) - oxl;
    const float ay = (r0.y - oyh) - oyl;
    const float az = (r0.z - ozh) - ozl;
    const float ux = r0.w, uy = r1.x, uz = r1.y, len = r1.z;
    A = make_float4(ax, ay, az, ux);
    B = make_float4(uy, uz, len, r1.w * c.inv_R4);
    uint64_t m = 0;
    const float inv_uz = uz > 1e-12f ? 1.0f / uz : 0.0f;
#pragma unroll 1
    for (int l = 0; l < nl; ++l) {
        const float zl = (float)l * c.fdz;
        float t_lo = 0.0f, t_hi = len;
        if (uz > 1e-12f) {
            t_lo = fmaxf((zl - c.cull - az) * inv_uz, 0.0f);
            t_hi = fminf((zl + c.cull - az) * inv_uz, len);
        } else if (fabsf(az - zl) > c.cull) {
            t_lo = 1.0f;
            t_hi = 0.0f;
        }
        if (t_lo <= t_hi) {
            const float xa = fmaf(t_lo, ux, ax), xb = fmaf(t_hi, ux, ax);
            const float ya = fmaf(t_lo, uy, ay), yb = fmaf(t_hi, uy, ay);
            const float xmin = fminf(xa, xb) - c.cull, xmax = fmaxf(xa, xb) + c.cull;
            const float ymin = fminf(ya, yb) - c.cull, ymax = fmaxf(ya, yb) + c.cull;
            const float qz = zl - az;
#pragma unroll
            for (int w = 0; w < kTileWarps; ++w) {
                const float rx0 = ((float)((w & 1) * 8) + 0.5f) * c.fpx;
                const float rx1 = ((float)((w & 1) * 8) + 7.5f) * c.fpx;
                const float ry0 = ((float)((w >> 1) * 4) + 0.5f) * c.fpx;
                const float ry1 = ((float)((w >> 1) * 4) + 3.5f) * c.fpx;
                if (xmax >= rx0 && xmin <= rx1 && ymax >= ry0 && ymin <= ry1) {
                    const float qx = 0.5f * (rx0 + rx1) - ax;
                    const float qy = 0.5f * (ry0 + ry1) - ay;
                    const float t = fmaf(qz, uz, fmaf(qy, uy, qx * ux));
                    const float ex = fmaf(-t, ux, qx), ey = fmaf(-t, uy, qy);
                    const float ez = fmaf(-t, uz, qz);
                    if (fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= c.cull_line2)
                        m |= 1ull << (w * 8 + l);
                }
            }
        }
    }
    return m;
}

// Loads record rp into tile-local coordinates (see stage_record).
__device__ __forceinline__ void load_record(const csl_rec* rp_rec, float oxh, float oxl, float oyh,
                                            float oyl, float ozh, float ozl, float inv_R4,
                                            float4& A, float4& B) {
    const float4* rp = reinterpret_cast<const float4*>(rp_rec);
    const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
    A = make_float4((r0.x - oxh) - oxl, (r0.y - oyh) - oyl, (r0.z - ozh) - ozl, r0.w);
    B = make_float4(r1.x, r1.y, r1.z, r1.w * inv_R4);
}

// Extent of a staged edge (A, B) in layer l of a 16 x 16 tile: the pixel rows
// j0..j1 and columns i0..i1 whose centres lie in the xy box of the edge clipped
// to |z - z_l| <= cull, grown by cull. Packed as j0 | j1 << 4 | i0 << 8 |
// i1 << 12 | 1 << 16; 0 when the box misses the tile or the layer.
__device__ __forceinline__ uint32_t item_extent(const float4 A, const float4 B, int l,
                                                const TileCull& c) {
    const float ax = A.x, ay = A.y, az = A.z, ux = A.w, uy = B.x, uz = B.y, len = B.z;
    const float zl = (float)l * c.fdz;
    float t_lo = 0.0f, t_hi = len;
    if (uz > 1e-12f) {
        const float inv_uz = 1.0f / uz;
        t_lo = fmaxf((zl - c.cull - az) * inv_uz, 0.0f);
        t_hi = fminf((zl + c.cull - az) * inv_uz, len);
    } else if (fabsf(az - zl) > c.cull) {
        return 0u;
    }
    if (t_lo > t_hi) return 0u;
    const float xa = fmaf(t_lo, ux, ax), xb = fmaf(t_hi, ux, ax);
    const float ya = fmaf(t_lo, uy, ay), yb = fmaf(t_hi, uy, ay);
    const float inv_px = 1.0f / c.fpx;
    // pixel i has its centre at (i + 1/2) px: i in [ceil(x_min/px - 1/2), floor(x_max/px - 1/2)]
    const float fx0 = fmaf(fminf(xa, xb) - c.cull, inv_px, -0.5f);
    const float fx1 = fmaf(fmaxf(xa, xb) + c.cull, inv_px, -0.5f);
    const float fy0 = fmaf(fminf(ya, yb) - c.cull, inv_px, -0.5f);
    const float fy1 = fmaf(fmaxf(ya, yb) + c.cull, inv_px, -0.5f);
    const int i0 = max(0, (int)ceilf(fmaxf(fx0, -1.0f)));
    const int i1 = min(15, (int)floorf(fminf(fx1, 16.0f)));
    const int j0 = max(0, (int)ceilf(fmaxf(fy0, -1.0f)));
    const int j1 = min(15, (int)floorf(fminf(fy1, 16.0f)));
    if (i0 > i1 || j0 > j1) return 0u;
    return (uint32_t)j0 | ((uint32_t)j1 << 4) | ((uint32_t)i0 << 8) | ((uint32_t)i1 << 12) |
           (1u << 16);
}

// Pixels i0..i1 of row j (within the extent e) whose centres lie within
// sqrt(r2) of the edge's line in plane zl (tile-local). The line meets the
// row's line {(x, y_j, zl)} at distance |Z u_y - Y u_z| / sqrt(a), a = u_y^2 +
// u_z^2, closest at X* = u_x (Y u_y + Z u_z) / a, and the squared distance
// grows as a (X - X*)^2, so the row's points within the radius are
// |X - X*| <= sqrt(r2 a - (Z u_y - Y u_z)^2) / a. Widened by 0.05 px. An edge
// along x (a ~ 0) keeps the extent's columns.
__device__ __forceinline__ bool row_span(const float4 A, const float4 B, float zl, int j,
                                         uint32_t e, const TileCull& c, float r2, int& i0,
                                         int& i1) {
    const float ux = A.w, uy = B.x, uz = B.y;
    i0 = (int)((e >> 8) & 15u);
    i1 = (int)((e >> 12) & 15u);
    const float a = fmaf(uy, uy, uz * uz);
    if (a > 1e-6f) {
        const float Y = fmaf((float)j, c.fpx, 0.5f * c.fpx) - A.y;
        const float Z = zl - A.z;
        const float dm = fmaf(Z, uy, -(Y * uz));
        const float q = fmaf(r2, a, -(dm * dm));
        if (q < 0.0f) return false;
        const float inv_a = 1.0f / a;
        const float xs = ux * fmaf(Y, uy, Z * uz) * inv_a + A.x;
        const float half = sqrt_approx(q) * inv_a;
        const float inv_px = 1.0f / c.fpx;
        const float f0 = fmaf(xs - half, inv_px, -0.55f);
        const float f1 = fmaf(xs + half, inv_px, -0.45f);
        i0 = max(i0, (int)ceilf(fmaxf(f0, -1.0f)));
        i1 = min(i1, (int)floorf(fminf(f1, 16.0f)));
    }
    return i0 <= i1;
}

// The warps of one layer l whose 8 x 4 block the staged edge (A, B) may reach
// (the test of stage_record for a single layer): bit w set for warp w.
__device__ __forceinline__ uint32_t cull_layer(const float4 A, const float4 B, int l,
                                               const TileCull& c) {
    const float ax = A.x, ay = A.y, az = A.z, ux = A.w, uy = B.x, uz = B.y, len = B.z;
    const float zl = (float)l * c.fdz;
    float t_lo = 0.0f, t_hi = len;
    if (uz > 1e-12f) {
        const float inv_uz = 1.0f / uz;
        t_lo = fmaxf((zl - c.cull - az) * inv_uz, 0.0f);
        t_hi = fminf((zl + c.cull - az) * inv_uz, len);
    } else if (fabsf(az - zl) > c.cull) {
        return 0u;
    }
    if (t_lo > t_hi) return 0u;
    const float xa = fmaf(t_lo, ux, ax), xb = fmaf(t_hi, ux, ax);
    const float ya = fmaf(t_lo, uy, ay), yb = fmaf(t_hi, uy, ay);
    const float xmin = fminf(xa, xb) - c.cull, xmax = fmaxf(xa, xb) + c.cull;
    const float ymin = fminf(ya, yb) - c.cull, ymax = fmaxf(ya, yb) + c.cull;
    const float qz = zl - az;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < kTileWarps; ++w) {
        const float rx0 = ((float)((w & 1) * 8) + 0.5f) * c.fpx;
        const float rx1 = ((float)((w & 1) * 8) + 7.5f) * c.fpx;
        const float ry0 = ((float)((w >> 1) * 4) + 0.5f) * c.fpx;
        const float ry1 = ((float)((w >> 1) * 4) + 3.5f) * c.fpx;
        if (xmax >= rx0 && xmin <= rx1 && ymax >= ry0 && ymin <= ry1) {
            const float qx = 0.5f * (rx0 + rx1) - ax;
            const float qy = 0.5f * (ry0 + ry1) - ay;
            const float t = fmaf(qz, uz, fmaf(qy, uy, qx * ux));
            const float ex = fmaf(-t, ux, qx), ey = fmaf(-t, uy, qy);
            const float ez = fmaf(-t, uz, qz);
            if (fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= c.cull_line2) m |= 1u << w;
        }
    }
    return m;
}

// Byte l of `bytes` holds the warp bits of layer l; returns warp w's layer
// bits (bit l = layer l).
__device__ __forceinline__ uint32_t warp_layers(uint64_t bytes, int w) {
    const uint64_t b = (bytes >> w) & 0x0101010101010101ull;
    return (uint32_t)((b * 0x0102040810204080ull) >> 56);
}

// In the frame of the edge: p - v_s = t0 u + e, h2 = max(R^2 - |e|^2, 0),
// w = sqrt(h2); the edge covers tau = t - t0 in [tau1, tau2] =
// [max(-t0, -w), min(L - t0, w)] and the kernel there is (h2 - tau^2)^2 / R^4.
// Returns R^4 I = integral of (h2 - tau^2)^2 over [tau1, tau2], by 3-point
// Gauss-Legendre (exact for this degree-4 polynomial, all terms >= 0). With
// m = (tau1 + tau2)/2, h = (tau2 - tau1)/2, c = h2 - m^2, A = c - 0.6 h^2 and
// B = 2 m h sqrt(0.6): R^4 I = h [(10/9)(A^2 + B^2) + (8/9) c^2].
__device__ __forceinline__ float segment_term_R4(float t0, float h2, float len) {
    const float w = sqrt_approx(h2);
    const float tau1 = fmaxf(-t0, -w);
    const float tau2 = fminf(len - t0, w);
    const float d = fmaxf(tau2 - tau1, 0.0f);   // 2 h
    const float s = tau2 + tau1;                 // 2 m
    const float cc = fmaf(-0.25f * s, s, h2);    // h2 - m^2
    const float d15 = 0.15f * d;
    const float Av = fmaf(-d15, d, cc);          // h2 - m^2 - 0.6 h^2
    const float ds = d15 * s;
    const float B2 = ds * (d * s);               // (2 m h sqrt(0.6))^2 = 0.15 d^2 s^2
    return d * fmaf(5.0f / 9.0f, fmaf(Av, Av, B2), (4.0f / 9.0f) * (cc * cc));
}

}  // namespace csl
