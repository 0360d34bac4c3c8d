// Field kernel: Sigma(p) = sum_j w_j I_j(p) (Eq. 6) on every pixel of a slab
// of S layers, one CTA per (slab, 16x16-pixel tile).
//
// I_j(p) is the integral of the quartic kernel (Eq. 5) along edge j by arc
// length (Eq. 7 with its Jacobian). In the frame of the edge, with
// p - v_s = t0 u + e (e orthogonal to u) and w^2 = R^2 - |e|^2, the kernel is
// (w^2 - tau^2)^2 / R^4 at tau = t - t0, and the edge covers
// tau in [tau1, tau2] = [max(-t0, -w), min(L - t0, w)]. The integrand is a
// polynomial of degree 4 in tau, so 3-point Gauss-Legendre on [tau1, tau2] is
// exact (it integrates degree <= 5 exactly); its terms are all >= 0, so FP32
// keeps a few-ulp relative error instead of the cancellation of the printed
// difference of quintics. With m = (tau1 + tau2)/2, h = (tau2 - tau1)/2,
// c = w^2 - m^2, A = c - 0.6 h^2 and B = 2 m h sqrt(0.6):
//   I R^4 = h [ (10/9)(A^2 + B^2) + (8/9) c^2 ].
//
// Coordinates are taken relative to the tile's corner (a double split into
// two floats), so no absolute pixel position ever rounds at the magnitude of
// the part (an ulp at 200 mm is 1.5e-5 mm, far above the 1e-5 relative field
// tolerance at strut surfaces).
//
// Work per CTA: the tile's edge list, which the binner stores contiguously (the
// records themselves, in list order), is staged into shared memory in chunks of
// 256 records by one bulk copy (TMA, cp.async.bulk) completed on an mbarrier;
// each thread converts its record to tile-local coordinates, then computes for
// every (record, layer) item whether the edge's support can reach each warp's
// 8x4-pixel block (xy box of the edge clipped to |z - z_layer| <= R, grown by
// R, and the block centre's distance to the line). Warps then walk only the
// records whose bit is set (ballot + ffs); the per-pixel evaluation is
// branch-free.
#include <math.h>

#include <vector>

#include "field_tile.cuh"
#include "slice.cuh"

namespace csl {
namespace {

struct FieldConst {
    int32_t nx, ny, ntx, n_tiles;
    int32_t n_layers;      // layers in this chunk
    int32_t first_layer;   // global index of the chunk's first layer
    double x0, y0, px, z0, dz;
    float R2, inv_R4, fpx, fdz, cull;
    float cull_line2;   // (cull + half-diagonal of a warp's pixel block)^2
    TileCull tc;        // the same values for stage_record
    float C;            // iso-value (inside mask)
    const float2* org_x;   // per tile column: x of its first pixel edge, (hi, lo)
    const float2* org_y;   // per tile row
    const float2* org_z;   // per slab: z of its first layer
    int32_t mwr;        // mask words per row
    int64_t mask_wpl;   // mask words per layer
    uint32_t* err;      // device status word: ST_TIMEOUT when a wait gave up
};

// One (tile, slab) of the field: called by the grid kernel (one CTA per
// (tile, slab)) and by the persistent batch kernel (one item at a time).
//
// The tile's records are contiguous (the binner copies them in list order), so
// each chunk of up to 256 records is staged by one bulk copy (TMA) issued by
// thread 0 and completed on an mbarrier; every thread then converts its record
// to tile-local coordinates in place. bar: the CTA's mbarrier (initialised
// with one arrival), phase: its parity, kept by the caller across tiles.
// Returns false (after setting ST_TIMEOUT in *c.err) when a copy never
// completed; the caller must then stop using the barrier.
template <int S, bool COUNT>
__device__ __forceinline__ bool field_tile(const csl_rec* __restrict__ recs,
                                           const uint32_t* __restrict__ tstart,
                                           const uint32_t* __restrict__ tend, const FieldConst& c,
                                           float* __restrict__ sigma, uint32_t* __restrict__ mask,
                                           unsigned long long* __restrict__ n_pairs, int tile,
                                           int slab, uint64_t* bar, uint32_t& phase) {
    __shared__ __align__(16) float4 s_rec[kFieldThreads][2];   // raw, then tile-local
    __shared__ uint64_t s_mask[kFieldThreads];   // byte l: warps reached at layer l

    const int tx = tile % c.ntx, ty = tile / c.ntx;
    const uint32_t key = (uint32_t)slab * (uint32_t)c.n_tiles + (uint32_t)tile;
    const uint32_t beg = tstart[key], end = tend[key];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = warp & 1, wy = warp >> 1;
    const int il = wx * 8 + (lane & 7), jl = wy * 4 + (lane >> 3);
    const int l0 = slab * S;
    const int nl = min(S, c.n_layers - l0);

    float acc[S];
#pragma unroll
    for (int l = 0; l < S; ++l) acc[l] = 0.0f;
    uint32_t n_nonzero = 0, n_eval = 0;

    if (end > beg) {
        // the tile's corner and the slab's first plane, each a (hi, lo) float pair
        const float2 ox = c.org_x[tx], oy = c.org_y[ty], oz = c.org_z[slab];
        const float oxh = ox.x, oxl = ox.y, oyh = oy.x, oyl = oy.y, ozh = oz.x, ozl = oz.y;
        const float pxl = ((float)il + 0.5f) * c.fpx;
        const float pyl = ((float)jl + 0.5f) * c.fpx;
        const TileCull cull = c.tc;

        for (uint32_t c0 = beg; c0 < end; c0 += kFieldThreads) {
            const int cnt = (int)min((uint32_t)kFieldThreads, end - c0);
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();   // the block's earlier reads of s_rec come first
                bulk_load(s_rec, recs + c0, (uint32_t)cnt * (uint32_t)sizeof(csl_rec), bar);
            }
            // a copy that never completes: report it, wait once more (bounded)
            // for the copy still in flight, and give the tile up
            if (__syncthreads_or(!mbar_wait(bar, phase))) {
                if (threadIdx.x == 0) atomicOr(c.err, ST_TIMEOUT);
                mbar_wait(bar, phase);
                return false;
            }
            phase ^= 1u;
            if ((int)threadIdx.x < cnt) {
                const float4 r0 = s_rec[threadIdx.x][0], r1 = s_rec[threadIdx.x][1];
                s_rec[threadIdx.x][0] =
                    make_float4((r0.x - oxh) - oxl, (r0.y - oyh) - oyl, (r0.z - ozh) - ozl, r0.w);
                s_rec[threadIdx.x][1] = make_float4(r1.x, r1.y, r1.z, r1.w * cull.inv_R4);
                s_mask[threadIdx.x] = 0;
            }
            __syncthreads();
            // cull masks: one (record, layer) item per thread; byte l of s_mask[r]
            // holds the warps of layer l
            for (int item = threadIdx.x; item < cnt * nl; item += kFieldThreads) {
                const int r = item % cnt, l = item / cnt;
                reinterpret_cast<uint8_t*>(s_mask)[8 * r + l] =
                    (uint8_t)cull_layer(s_rec[r][0], s_rec[r][1], l, cull);
            }
            __syncthreads();
            for (int i0 = 0; i0 < cnt; i0 += 32) {
                const int i = i0 + lane;
                const uint32_t wm = i < cnt ? warp_layers(s_mask[i], warp) : 0u;
                uint32_t ball = __ballot_sync(0xffffffffu, wm != 0u);
                while (ball) {
                    const int b = __ffs(ball) - 1;
                    ball &= ball - 1u;
                    const uint32_t lm = __shfl_sync(0xffffffffu, wm, b);
                    const float4 A = s_rec[i0 + b][0], B = s_rec[i0 + b][1];
                    const float dx = pxl - A.x, dy = pyl - A.y;
                    const float txy = fmaf(dy, B.x, dx * A.w);
#pragma unroll
                    for (int l = 0; l < S; ++l) {
                        if (lm & (1u << l)) {
                            const float dz = (float)l * c.fdz - A.z;
                            const float t0 = fmaf(dz, B.y, txy);
                            const float ex = fmaf(-t0, A.w, dx);
                            const float ey = fmaf(-t0, B.x, dy);
                            const float ez = fmaf(-t0, B.y, dz);
                            const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                            const float h2 = fmaxf(c.R2 - d2, 0.0f);
                            // the rest only when some pixel of the warp is within R
                            if (__any_sync(0xffffffffu, h2 > 0.0f)) {
                                const float I = segment_term_R4(t0, h2, B.z);
                                acc[l] = fmaf(B.w, I, acc[l]);
                                if (COUNT) {
                                    n_nonzero += I > 0.0f;
                                    ++n_eval;
                                }
                            }
                        }
                    }
                }
            }
            // the next chunk reuses s_rec and s_mask; after the last one each warp
            // goes on to its own pixels without waiting (a persistent caller
            // synchronises before the next item)
            if (c0 + (uint32_t)kFieldThreads < end) __syncthreads();
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
    const int gi = tx * kTile + il, gj = ty * kTile + jl;
    const bool in_grid = gi < c.nx && gj < c.ny;
    if (in_grid && sigma) {   // no Sigma plane when only the mask is wanted
#pragma unroll
        for (int l = 0; l < S; ++l)
            if (l < nl) sigma[((int64_t)(l0 + l) * c.ny + gj) * c.nx + gi] = acc[l];
    }
    if (mask) {
        // inside bits of the warp's 8 x 4 block: one byte per pixel row, OR-ed
        // into the padded row (pixel i is padded sample i + 1)
        const int I0 = tx * kTile + wx * 8 + 1;
        const int sh = I0 & 31;
#pragma unroll
        for (int l = 0; l < S; ++l) {
            if (l >= nl) break;
            const uint32_t ball = __ballot_sync(0xffffffffu, in_grid && acc[l] >= c.C);
            if (lane < 4) {
                const uint32_t byte = (ball >> (8 * lane)) & 0xffu;
                if (byte) {
                    const int J = ty * kTile + wy * 4 + lane + 1;
                    uint32_t* row = mask + (int64_t)(l0 + l) * c.mask_wpl + (int64_t)J * c.mwr;
                    atomicOr(row + (I0 >> 5), byte << sh);
                    const uint32_t hi = sh > 24 ? byte >> (32 - sh) : 0u;
                    if (hi) atomicOr(row + (I0 >> 5) + 1, hi);
                }
            }
        }
    }
    return true;
}

template <int S, bool COUNT>
__global__ void __launch_bounds__(kFieldThreads, 8)
k_field(const csl_rec* __restrict__ recs, const uint32_t* __restrict__ tstart,
        const uint32_t* __restrict__ tend, FieldConst c, float* __restrict__ sigma,
        uint32_t* __restrict__ mask, unsigned long long* __restrict__ n_pairs) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    field_tile<S, COUNT>(recs, tstart, tend, c, sigma, mask, n_pairs, blockIdx.x, blockIdx.y,
                         &bar, phase);
}

// One job of a batch, as the persistent kernel reads it.
struct FieldJob {
    FieldConst c;
    const csl_rec* recs;   // the binned records, in list order
    const uint32_t* tstart;
    const uint32_t* tend;
    float* sigma;
    uint32_t* mask;
};
static_assert(sizeof(FieldJob) % 4 == 0, "FieldJob is copied as 32-bit words");

// Persistent field kernel over the (job, slab, tile) items of a batch: each
// CTA takes the next item from a shared counter, in the order `order` gives
// (longest tile lists first, so the short ones fill the tail).
template <int S>
__global__ void __launch_bounds__(kFieldThreads, 6)
k_field_batch(const FieldJob* __restrict__ jobs, const uint2* __restrict__ items,
              const uint32_t* __restrict__ order, uint32_t n_items, uint32_t* counter) {
    __shared__ uint32_t s_item;
    __shared__ FieldJob s_job;
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
            for (int i = threadIdx.x; i < (int)(sizeof(FieldJob) / 4); i += kFieldThreads)
                reinterpret_cast<uint32_t*>(&s_job)[i] = src[i];
            __syncthreads();
        }
        const uint32_t n_tiles = (uint32_t)s_job.c.n_tiles;
        if (!field_tile<S, false>(s_job.recs, s_job.tstart, s_job.tend, s_job.c, s_job.sigma,
                                  s_job.mask, nullptr, (int)(item.y % n_tiles),
                                  (int)(item.y / n_tiles), &bar, phase))
            break;   // a bulk copy gave up (reported): this CTA takes no more items
        __syncthreads();   // shared memory is reused by the next item
    }
}

// The field kernel's bounded mbarrier wait on a barrier that nothing arms: it
// must give up after `polls` polls and report ST_TIMEOUT (test of the path).
__global__ void k_wait_nothing(uint32_t polls, uint32_t* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait(&bar, 0, polls)) && threadIdx.x == 0) atomicOr(err, ST_TIMEOUT);
}

// items[i] = (job, slab * n_tiles + tile) for the jobs' item ranges off[j]..off[j+1].
__global__ void k_make_items(const int64_t* __restrict__ off, int n_jobs, uint2* __restrict__ items) {
    const int64_t n = off[n_jobs];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_jobs - 1;   // the last job with off[j] <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        items[i] = make_uint2((uint32_t)lo, (uint32_t)(i - off[lo]));
    }
}

// Sort keys for the item queue: longest tile list first (16-bit key).
__global__ void k_item_keys(const FieldJob* __restrict__ jobs, const uint2* __restrict__ items,
                            uint32_t n, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint2 it = items[i];
        const FieldJob& J = jobs[it.x];
        const uint32_t len = J.tend[it.y] - J.tstart[it.y];
        keys[i] = 0xffffu - min(len, 0xffffu);
        vals[i] = i;
    }
}

// Corner of each tile column / row and first plane of each slab, computed in
// double (non-fused) and split into a (hi, lo) float pair.
__global__ void k_origins(float2* __restrict__ org, int ntx, int nty, int n_slabs, double x0,
                          double y0, double z0, double px, double dz, int first_layer, int S,
                          int T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v;
    if (i < ntx) v = __dadd_rn(x0, __dmul_rn((double)(i * T), px));
    else if (i < ntx + nty) v = __dadd_rn(y0, __dmul_rn((double)((i - ntx) * T), px));
    else if (i < ntx + nty + n_slabs)
        v = __dadd_rn(z0, __dmul_rn((double)(first_layer + (i - ntx - nty) * S), dz));
    else return;
    const float hi = (float)v;
    org[i] = make_float2(hi, (float)__dsub_rn(v, (double)hi));
}

}  // namespace

namespace {

// Kernel constants of a chunk; org = the chunk's origin tables (ntx + nty +
// n_slabs float2, as k_origins writes them).
FieldConst make_field_const(const ChunkGeom& g, float C, const float2* org) {
    FieldConst c;
    c.C = C;
    c.org_x = org;
    c.org_y = org + g.ntx;
    c.org_z = org + g.ntx + g.nty;
    c.mwr = (int32_t)mask_words_per_row(g.nx);
    c.mask_wpl = mask_words_per_layer(g.nx, g.ny);
    c.nx = g.nx;
    c.ny = g.ny;
    c.ntx = g.ntx;
    c.n_tiles = g.ntx * g.nty;
    c.n_layers = g.n_layers;
    c.first_layer = g.first_layer;
    c.x0 = g.x0;
    c.y0 = g.y0;
    c.px = g.px;
    c.z0 = g.z0;
    c.dz = g.dz;
    c.R2 = (float)(g.R * g.R);
    c.inv_R4 = (float)(1.0 / (g.R * g.R * g.R * g.R));
    c.fpx = (float)g.px;
    c.fdz = (float)g.dz;
    c.cull = (float)(g.R * (1.0 + 1e-5) + 1e-6);
    {
        // pixel centres of a warp's 8 x 4 block lie within 3.5 x 1.5 pixels of its centre
        double hd = g.px * sqrt(3.5 * 3.5 + 1.5 * 1.5) * (1.0 + 1e-5);
        double r = (double)c.cull + hd;
        c.cull_line2 = (float)(r * r);
    }
    c.tc.fpx = c.fpx;
    c.tc.fdz = c.fdz;
    c.tc.cull = c.cull;
    c.tc.cull_line2 = c.cull_line2;
    c.tc.inv_R4 = c.inv_R4;
    return c;
}

void launch_origins(const ChunkGeom& g, float2* org, cudaStream_t s) {
    k_origins<<<(unsigned)ceil_div(g.ntx + g.nty + g.n_slabs, 128), 128, 0, s>>>(
        org, g.ntx, g.nty, g.n_slabs, g.x0, g.y0, g.z0, g.px, g.dz, g.first_layer, g.S, g.T);
    CSL_LAUNCH_CHECK("origins");
}

}  // namespace

void field_chunk(const csl_lattice* L, const ChunkGeom& g, const SlabBins& bins, float C,
                 float* sigma, uint32_t* mask, unsigned long long* count_pairs, cudaStream_t s,
                 FusedVerts* fv) {
    // tile and slab origins in double, each split into a (hi, lo) float pair
    DevBuf org_d(((size_t)g.ntx + g.nty + g.n_slabs) * sizeof(float2), s);
    launch_origins(g, org_d.as<float2>(), s);
    if (g.kernel == kFieldFootprint) {
        field_chunk_fp(g, bins, C, org_d.as<float2>(), L->status.as<uint32_t>(), sigma, mask,
                       count_pairs, s, fv);
        return;
    }
    if (g.fused || fv) fail(CSL_ERR_INVALID_ARG, "the fused pass needs the footprint kernel");
    if (g.T != kTile) fail(CSL_ERR_INVALID_ARG, "the block field kernel takes 16-pixel tiles");
    FieldConst c = make_field_const(g, C, org_d.as<float2>());
    c.err = L->status.as<uint32_t>();
    dim3 grid((unsigned)c.n_tiles, (unsigned)g.n_slabs);
    const csl_rec* recs = bins.recs.as<csl_rec>();
    const uint32_t* ts = bins.tile_start.as<uint32_t>();
    const uint32_t* te = bins.tile_end.as<uint32_t>();
#define CSL_FIELD_CASE(SV)                                                                    \
    case SV:                                                                                  \
        if (count_pairs)                                                                      \
            k_field<SV, true><<<grid, kFieldThreads, 0, s>>>(recs, ts, te, c, sigma, mask,    \
                                                             count_pairs);                    \
        else                                                                                  \
            k_field<SV, false><<<grid, kFieldThreads, 0, s>>>(recs, ts, te, c, sigma, mask,   \
                                                              nullptr);                       \
        break;
    switch (g.S) {
        CSL_FIELD_CASE(1)
        CSL_FIELD_CASE(2)
        CSL_FIELD_CASE(4)
        CSL_FIELD_CASE(8)
        default: fail(CSL_ERR_INVALID_ARG, "slab depth must be 1, 2, 4 or 8");
    }
#undef CSL_FIELD_CASE
    CSL_LAUNCH_CHECK("field");
}

void field_batch_prepare(const std::vector<FieldBatchJob>& jobs, FieldBatch& fb, cudaStream_t s) {
    const int n_jobs = (int)jobs.size();
    if (n_jobs == 0) fail(CSL_ERR_INVALID_ARG, "empty batch");
    const int S = jobs[0].g.S;
    const int kern = jobs[0].g.kernel, T = jobs[0].g.T, K = jobs[0].g.K;
    size_t n_org = 0;
    std::vector<int64_t> off(n_jobs + 1, 0);
    for (int j = 0; j < n_jobs; ++j) {
        const ChunkGeom& g = jobs[j].g;
        if (g.S != S) fail(CSL_ERR_INVALID_ARG, "batch: one slab depth for every job");
        if (g.kernel != kern || g.T != T || g.K != K || g.fused)
            fail(CSL_ERR_INVALID_ARG, "batch: one field kernel, tile and staging chunk");
        if (kern == kFieldBlock && T != kTile)
            fail(CSL_ERR_INVALID_ARG, "batch: the block field kernel takes 16-pixel tiles");
        n_org += (size_t)g.ntx + g.nty + g.n_slabs;
        off[j + 1] = off[j] + (int64_t)g.n_slabs * g.ntx * g.nty;
    }
    if (off[n_jobs] >= 0xffffffffLL) fail(CSL_ERR_CAPACITY, "batch: more than 2^32 - 1 tiles");
    fb.S = S;
    fb.kernel = kern;
    fb.T = T;
    fb.K = K;
    fb.n_items = off[n_jobs];
    fb.origins.alloc_persistent(n_org * sizeof(float2));
    std::vector<FieldJob> hj(n_jobs);
    std::vector<const float2*> orgs(n_jobs);
    size_t o = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const FieldBatchJob& J = jobs[j];
        float2* org = fb.origins.as<float2>() + o;
        orgs[j] = org;
        launch_origins(J.g, org, s);
        o += (size_t)J.g.ntx + J.g.nty + J.g.n_slabs;
        hj[j].c = make_field_const(J.g, (float)J.L->C, org);
        hj[j].c.err = J.err;
        hj[j].recs = J.bins->recs.as<csl_rec>();
        hj[j].tstart = J.bins->tile_start.as<uint32_t>();
        hj[j].tend = J.bins->tile_end.as<uint32_t>();
        hj[j].sigma = J.sigma;
        hj[j].mask = J.mask;
    }
    fb.jobs.alloc_persistent(sizeof(FieldJob) * n_jobs);
    DevBuf off_d((size_t)(n_jobs + 1) * 8, s);
    CSL_CUDA(cudaMemcpyAsync(fb.jobs.get(), hj.data(), sizeof(FieldJob) * n_jobs,
                             cudaMemcpyHostToDevice, s));
    std::vector<unsigned char> hfp;
    if (kern == kFieldFootprint) {
        fp_batch_jobs(jobs, orgs.data(), hfp);
        fb.fp_jobs.alloc_persistent(hfp.size());
        CSL_CUDA(cudaMemcpyAsync(fb.fp_jobs.get(), hfp.data(), hfp.size(),
                                 cudaMemcpyHostToDevice, s));
    }
    CSL_CUDA(cudaMemcpyAsync(off_d.get(), off.data(), (size_t)(n_jobs + 1) * 8,
                             cudaMemcpyHostToDevice, s));
    const size_t n = (size_t)fb.n_items;
    fb.items.alloc_persistent(n * sizeof(uint2));
    fb.keys.alloc_persistent(n * 4);
    fb.vals.alloc_persistent(n * 4);
    fb.tmp_keys.alloc_persistent(n * 4);
    fb.tmp_vals.alloc_persistent(n * 4);
    fb.counter.alloc_persistent(4);
    k_make_items<<<grid_for(fb.n_items, 256), 256, 0, s>>>(off_d.as<int64_t>(), n_jobs,
                                                          fb.items.as<uint2>());
    CSL_LAUNCH_CHECK("batch items");
    CSL_CUDA(cudaStreamSynchronize(s));   // the host tables above go out of scope
}

void field_batch_run(FieldBatch& fb, int n_ctas, cudaStream_t s) {
    if (fb.n_items == 0) return;
    const uint32_t n = (uint32_t)fb.n_items;
    k_item_keys<<<grid_for(fb.n_items, 256), 256, 0, s>>>(
        fb.jobs.as<FieldJob>(), fb.items.as<uint2>(), n, fb.keys.as<uint32_t>(),
        fb.vals.as<uint32_t>());
    CSL_LAUNCH_CHECK("batch item keys");
    radix_sort_pairs(fb.keys.as<uint32_t>(), fb.vals.as<uint32_t>(), fb.tmp_keys.as<uint32_t>(),
                     fb.tmp_vals.as<uint32_t>(), fb.n_items, 16, s);
    CSL_CUDA(cudaMemsetAsync(fb.counter.get(), 0, 4, s));
    const FieldJob* jobs = fb.jobs.as<FieldJob>();
    const uint2* items = fb.items.as<uint2>();
    const uint32_t* order = fb.vals.as<uint32_t>();
    uint32_t* counter = fb.counter.as<uint32_t>();
    if (fb.kernel == kFieldFootprint) {
        fp_batch_launch(fb.fp_jobs.get(), items, order, n, counter, fb.T, fb.S, fb.K, n_ctas, s);
        return;
    }
    switch (fb.S) {
        case 1: k_field_batch<1><<<n_ctas, kFieldThreads, 0, s>>>(jobs, items, order, n, counter); break;
        case 2: k_field_batch<2><<<n_ctas, kFieldThreads, 0, s>>>(jobs, items, order, n, counter); break;
        case 4: k_field_batch<4><<<n_ctas, kFieldThreads, 0, s>>>(jobs, items, order, n, counter); break;
        case 8: k_field_batch<8><<<n_ctas, kFieldThreads, 0, s>>>(jobs, items, order, n, counter); break;
        default: fail(CSL_ERR_INVALID_ARG, "slab depth must be 1, 2, 4 or 8");
    }
    CSL_LAUNCH_CHECK("batch field");
}

}  // namespace csl

extern "C" csl_status csl_debug_wait_timeout(uint32_t polls, void* stream) {
    try {
        if (polls == 0 || polls > csl::kWaitLimit) csl::fail(CSL_ERR_INVALID_ARG, "polls in [1, 2^22]");
        cudaStream_t s = (cudaStream_t)stream;
        csl::DevBuf err(4, s);
        CSL_CUDA(cudaMemsetAsync(err.get(), 0, 4, s));
        csl::k_wait_nothing<<<1, 64, 0, s>>>(polls, err.as<uint32_t>());
        CSL_LAUNCH_CHECK("wait test");
        uint32_t st = 0;
        csl::read_to_host(&st, err.get(), 4, s);
        if (st & csl::ST_TIMEOUT) csl::fail(CSL_ERR_TIMEOUT, "the wait gave up as it should");
        return CSL_OK;
    } catch (const csl::Error& e) {
        csl::set_last_error(e.what());
        return e.code;
    } catch (...) {
        csl::set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}
