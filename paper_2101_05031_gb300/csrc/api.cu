// C ABI entry points and the streamed slicing driver (Sec. 4): the layers are
// processed in chunks; per chunk the binner, the field kernel and the contour
// kernels run on the caller's stream, and the chunk's contours are appended
// to the result.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <new>

#include "slice.cuh"

using namespace csl;

namespace csl {

void require_device_resident(const csl_lattice* L) {
    if (L && L->host_resident)
        fail(CSL_ERR_NOT_READY,
             "the lattice is host-resident (csl_lattice_upload_streamed): only slicing streams it");
}

void require_arg(bool ok, const char* msg) {
    if (!ok) fail(CSL_ERR_INVALID_ARG, msg);
}

// Resolves tile / slab / chunk sizes and the rounding margins of the binner.
SlicePlan make_plan(const csl_lattice* L, const csl_slice_desc& d) {
    require_arg(d.tile == 0 || d.tile == 16 || d.tile == 32, "tile must be 0, 16 or 32");
    require_arg(d.field_kernel == CSL_FIELD_AUTO || d.field_kernel == CSL_FIELD_BLOCK ||
                    d.field_kernel == CSL_FIELD_FOOTPRINT,
                "field_kernel must be CSL_FIELD_AUTO, CSL_FIELD_BLOCK or CSL_FIELD_FOOTPRINT");
    require_arg(d.stage_records == 0 ||
                    (d.stage_records >= 32 && d.stage_records <= 1024 && d.stage_records % 32 == 0),
                "stage_records must be 0 or a multiple of 32 up to 1024");
    SlicePlan p;
    // the footprint kernel where the support is a few pixels across (its lanes
    // follow the support), the block kernel where it covers whole blocks
    int kernel = d.field_kernel;
    if (kernel == CSL_FIELD_AUTO)
        kernel = (d.tile != 16 && L->R < 10.0 * d.pixel) ? CSL_FIELD_FOOTPRINT : CSL_FIELD_BLOCK;
    require_arg(kernel == CSL_FIELD_FOOTPRINT || d.tile != 32,
                "32-pixel tiles need the footprint field kernel");
    p.kernel = kernel == CSL_FIELD_FOOTPRINT ? kFieldFootprint : kFieldBlock;
    p.T = d.tile ? d.tile : (p.kernel == kFieldFootprint ? 32 : 16);
    p.K = d.stage_records ? d.stage_records : 256;
    int S = d.slab;
    if (S == 0) S = d.n_layers >= 8 ? 8 : (d.n_layers >= 4 ? 4 : (d.n_layers >= 2 ? 2 : 1));
    require_arg(S == 1 || S == 2 || S == 4 || S == 8, "slab must be 0, 1, 2, 4 or 8");
    p.S = S;
    p.ntx = (int)ceil_div(d.nx, p.T);
    p.nty = (int)ceil_div(d.ny, p.T);
    const int64_t plane = (int64_t)d.nx * d.ny;
    int chunk = d.chunk_layers;
    if (chunk == 0) {
        // about 4 GiB of Sigma per chunk (fewer launches and read-backs per
        // layer than smaller chunks); whole slabs, at least one slab
        int64_t c = ((int64_t)4 << 30) / (4 * plane);
        c = std::max<int64_t>(S, c - c % S);
        c = std::min<int64_t>(c, std::max(d.n_layers, 1));
        chunk = (int)c;
    }
    require_arg(chunk > 0 && (chunk % S == 0 || chunk >= d.n_layers),
            "chunk_layers must be a positive multiple of the slab depth");
    // marching squares needs < 2^27 edge words per chunk
    const int64_t words_per_layer = 2 * mask_words_per_layer(d.nx, d.ny);
    if ((int64_t)chunk * words_per_layer >= ((int64_t)1 << 27)) {
        int64_t c = (((int64_t)1 << 27) - 1) / words_per_layer;
        c -= c % S;
        require_arg(c >= S, "grid too large for one slab per chunk");
        chunk = (int)c;
    }
    p.chunk = chunk;
    double scale = 1.0;
    for (int k = 0; k < 3; ++k)
        scale = std::max({scale, fabs((double)L->bbox_lo[k]), fabs((double)L->bbox_hi[k])});
    scale = std::max({scale, fabs(d.x0), fabs(d.y0), fabs(d.x0 + d.nx * d.pixel),
                      fabs(d.y0 + d.ny * d.pixel), fabs(d.z0),
                      fabs(d.z0 + (double)std::max(d.n_layers - 1, 0) * d.dz)});
    p.margin = (float)(L->R + 8e-6 * scale + 1e-6);
    return p;
}

bool wants_fused(const csl_slice_desc& d, const SlicePlan& p) {
    return p.kernel == kFieldFootprint && !(d.flags & CSL_SLICE_NO_CONTOURS) &&
           (d.flags & CSL_SLICE_FUSED);
}

ChunkGeom chunk_geom(const csl_lattice* L, const csl_slice_desc& d, const SlicePlan& p, int first,
                     int n) {
    ChunkGeom g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.ntx = p.ntx;
    g.nty = p.nty;
    g.x0 = d.x0;
    g.y0 = d.y0;
    g.px = d.pixel;
    g.z0 = d.z0;
    g.dz = d.dz;
    g.first_layer = first;
    g.n_layers = n;
    g.S = p.S;
    g.n_slabs = (int)ceil_div(n, p.S);
    g.R = L->R;
    g.margin_xy = p.margin;
    g.margin_z = p.margin;
    g.T = p.T;
    g.kernel = p.kernel;
    g.K = p.K;
    g.fused = p.fused;
    return g;
}

void check_lattice_status(const csl_lattice* L, cudaStream_t s) {
    uint32_t st = 0;
    read_to_host(&st, L->status.get(), 4, s);
    if (st) {
        CSL_CUDA(cudaMemsetAsync(L->status.get(), 0, 4, s));
        CSL_CUDA(cudaStreamSynchronize(s));
        fail(CSL_ERR_TIMEOUT, "a device wait (bulk copy of the field kernel) gave up");
    }
}

void validate_desc(const csl_slice_desc* d) {
    require_arg(d != nullptr, "desc is NULL");
    require_arg(d->n_layers >= 0, "n_layers < 0");
    require_arg(d->nx >= 1 && d->ny >= 1 && d->nx <= 32000 && d->ny <= 32000,
            "nx, ny must be in [1, 32000]");
    require_arg(isfinite(d->pixel) && d->pixel > 0, "pixel must be > 0");
    require_arg(isfinite(d->x0) && isfinite(d->y0) && isfinite(d->z0), "non-finite origin");
    // layer k lies at z0 + k dz, so a non-finite dz poisons even a single layer
    require_arg(isfinite(d->dz), "dz must be finite");
    require_arg(d->n_layers <= 1 || d->dz > 0, "dz must be > 0");
}

}  // namespace csl

namespace {

thread_local csl_stats t_stats = {};

csl_status guard(const std::function<void()>& f) {
    try {
        f();
        return CSL_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return CSL_ERR_OOM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return CSL_ERR_CUDA;
    } catch (...) {
        set_last_error("unknown error");
        return CSL_ERR_CUDA;
    }
}

void require(bool ok, const char* msg) {
    if (!ok) fail(CSL_ERR_INVALID_ARG, msg);
}

void copy_in(DevBuf& dst, const void* src, size_t bytes, bool on_device, cudaStream_t s) {
    dst.ensure_persistent(bytes);
    if (bytes == 0) return;
    CSL_CUDA(cudaMemcpyAsync(dst.get(), src, bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

// The inside mask without its padding ring: out[(k * ny + j) * wpr + w] holds
// pixels 32 w .. 32 w + 31 of row j of layer k; in the padded mask, pixel i of
// row j is bit i + 1 of row j + 1 (the ring bits are 0, so bits past nx are 0).
__global__ void k_unpad_mask(const uint32_t* __restrict__ pad, int nx, int ny, int n_layers,
                             int64_t mwr, int64_t mask_wpl, uint32_t* __restrict__ out) {
    const int64_t wpr = (nx + 31) / 32;
    const int64_t n = (int64_t)n_layers * ny * wpr;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = t % wpr, row = t / wpr;
        const int64_t j = row % ny, k = row / ny;
        const uint32_t* pr = pad + k * mask_wpl + (j + 1) * mwr;
        const uint32_t lo = pr[w] >> 1;
        const uint32_t hi = w + 1 < mwr ? pr[w + 1] << 31 : 0u;
        out[t] = lo | hi;
    }
}

__global__ void k_add_i64(int64_t* a, int64_t n, int64_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] += v;
}

}  // namespace

extern "C" {

const char* csl_last_error(void) { return last_error_cstr(); }
const char* csl_version(void) { return "cslice 0.1 (sm_103a)"; }

csl_status csl_last_stats(csl_stats* out) {
    return guard([&] {
        require(out != nullptr, "out is NULL");
        *out = t_stats;
    });
}

csl_status csl_lattice_upload(const float* nodes_xyz, int64_t n_nodes, const int32_t* edges_ij,
                              const float* radius, int64_t n_edges, const csl_params* params,
                              void* stream, csl_lattice** out) {
    return guard([&] {
        require(out != nullptr, "out is NULL");
        *out = nullptr;
        require(n_nodes >= 0 && n_edges >= 0, "negative size");
        require(n_edges <= 0x7fffffffLL && n_nodes <= 0x7fffffffLL, "more than 2^31 - 1 items");
        require(n_nodes == 0 || nodes_xyz != nullptr, "nodes_xyz is NULL");
        require(n_edges == 0 || (edges_ij != nullptr && radius != nullptr),
                "edges_ij or radius is NULL");
        csl_params p = {0.0, 1.0, CSL_MODE_PHYSICAL, 0};
        if (params) p = *params;
        if (p.C == 0.0) p.C = 1.0;
        require(isfinite(p.C) && p.C > 0, "C must be > 0");
        require(p.mode == CSL_MODE_PHYSICAL || p.mode == CSL_MODE_RAW, "unknown mode");
        require(isfinite(p.R), "R must be finite");
        cudaStream_t s = (cudaStream_t)stream;
        csl_lattice* L = new csl_lattice();
        try {
            L->n_nodes = n_nodes;
            L->n_edges = n_edges;
            L->R = p.R;
            L->C = p.C;
            L->mode = p.mode;
            bool dev = p.input_on_device != 0;
            copy_in(L->nodes, nodes_xyz, (size_t)n_nodes * 12, dev, s);
            copy_in(L->edges, edges_ij, (size_t)n_edges * 8, dev, s);
            copy_in(L->radius, radius, (size_t)n_edges * 4, dev, s);
            L->status.alloc_persistent(4);
            CSL_CUDA(cudaMemsetAsync(L->status.get(), 0, 4, s));
            prepare_lattice(L, true, s);
            CSL_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            delete L;
            throw;
        }
        *out = L;
    });
}

csl_status csl_lattice_upload_streamed(const float* nodes_xyz, int64_t n_nodes,
                                       const int32_t* edges_ij, const float* radius,
                                       int64_t n_edges, const csl_params* params,
                                       int64_t batch_edges, void* stream, csl_lattice** out) {
    return guard([&] {
        require(out != nullptr, "out is NULL");
        *out = nullptr;
        require(n_nodes >= 0 && n_edges >= 0, "negative size");
        require(n_edges <= 0x7fffffffLL && n_nodes <= 0x7fffffffLL, "more than 2^31 - 1 items");
        require(n_nodes == 0 || nodes_xyz != nullptr, "nodes_xyz is NULL");
        require(n_edges == 0 || (edges_ij != nullptr && radius != nullptr),
                "edges_ij or radius is NULL");
        require(batch_edges >= 0, "batch_edges must be >= 0");
        csl_params p = {0.0, 1.0, CSL_MODE_PHYSICAL, 0};
        if (params) p = *params;
        require(p.input_on_device == 0, "a streamed lattice takes host arrays");
        if (p.C == 0.0) p.C = 1.0;
        require(isfinite(p.C) && p.C > 0, "C must be > 0");
        require(p.mode == CSL_MODE_PHYSICAL || p.mode == CSL_MODE_RAW, "unknown mode");
        require(isfinite(p.R), "R must be finite");
        cudaStream_t s = (cudaStream_t)stream;
        csl_lattice* L = new csl_lattice();
        try {
            L->n_nodes = n_nodes;
            L->n_edges = n_edges;
            L->R = p.R;
            L->C = p.C;
            L->mode = p.mode;
            copy_in(L->nodes, nodes_xyz, (size_t)n_nodes * 12, false, s);
            L->status.alloc_persistent(4);
            CSL_CUDA(cudaMemsetAsync(L->status.get(), 0, 4, s));
            prepare_lattice_streamed(L, edges_ij, radius,
                                     batch_edges > 0 ? batch_edges : ((int64_t)1 << 24), s);
            CSL_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            delete L;
            throw;
        }
        *out = L;
    });
}

csl_status csl_lattice_update(csl_lattice* L, const float* nodes_xyz, const float* radius,
                              void* stream) {
    return guard([&] {
        require(L != nullptr, "lattice is NULL");
        require_device_resident(L);
        cudaStream_t s = (cudaStream_t)stream;
        if (nodes_xyz && L->n_nodes > 0)
            CSL_CUDA(cudaMemcpyAsync(L->nodes.get(), nodes_xyz, (size_t)L->n_nodes * 12,
                                     cudaMemcpyDeviceToDevice, s));
        if (radius && L->n_edges > 0)
            CSL_CUDA(cudaMemcpyAsync(L->radius.get(), radius, (size_t)L->n_edges * 4,
                                     cudaMemcpyDeviceToDevice, s));
        prepare_lattice(L, false, s);
        CSL_CUDA(cudaStreamSynchronize(s));
    });
}

csl_status csl_lattice_get_info(const csl_lattice* L, csl_lattice_info* out) {
    return guard([&] {
        require(L != nullptr && out != nullptr, "NULL argument");
        memset(out, 0, sizeof(*out));
        out->n_nodes = L->n_nodes;
        out->n_edges = L->n_edges;
        out->R = L->R;
        out->C = L->C;
        out->mode = L->mode;
        for (int k = 0; k < 3; ++k) { out->bbox_lo[k] = L->bbox_lo[k]; out->bbox_hi[k] = L->bbox_hi[k]; }
        out->max_dz = L->max_dz;
        out->max_radius = L->max_radius;
    });
}

void csl_lattice_free(csl_lattice* L) { delete L; }

void csl_contours_free(csl_contours* c) {
    if (!c) return;
    if (c->on_device) {   // arrays grown in place (slicing) go back through their registry
        for (void* p : {(void*)c->layer_loop_off, (void*)c->loop_vert_off, (void*)c->xy,
                        (void*)c->edge_id})
            if (p && !growmap_free(p)) cudaFree(p);
    } else {
        host_block_free(c->layer_loop_off);   // offsets block
        host_block_free(c->xy);               // vertex block (edge ids included)
    }
    delete c;
}

csl_status csl_contours_copy(const csl_contours* c, int64_t* layer_loop_off,
                             int64_t* loop_vert_off, float* xy, int32_t* edge_id,
                             int32_t dst_on_device, void* stream) {
    return guard([&] {
        require(c != nullptr, "contours is NULL");
        require(!edge_id || c->edge_id, "these contours carry no edge ids");
        cudaStream_t s = (cudaStream_t)stream;
        cudaMemcpyKind kind = c->on_device ? (dst_on_device ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyDeviceToHost)
                                           : (dst_on_device ? cudaMemcpyHostToDevice
                                                            : cudaMemcpyHostToHost);
        auto cp = [&](void* dst, const void* src, size_t bytes) {
            if (dst && bytes) CSL_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
        };
        cp(layer_loop_off, c->layer_loop_off, (size_t)(c->n_layers + 1) * 8);
        cp(loop_vert_off, c->loop_vert_off, (size_t)(c->n_loops + 1) * 8);
        cp(xy, c->xy, (size_t)c->n_verts * 8);
        cp(edge_id, c->edge_id, (size_t)c->n_verts * 4);
        CSL_CUDA(cudaStreamSynchronize(s));
    });
}

csl_status csl_contours_create(int32_t n_layers, int64_t n_loops, int64_t n_verts,
                               const int64_t* layer_loop_off, const int64_t* loop_vert_off,
                               const float* xy, const int32_t* edge_id, void* stream,
                               csl_contours** out) {
    csl_contours* c = nullptr;
    const csl_status st = guard([&] {
        require(out != nullptr, "out is NULL");
        *out = nullptr;
        require(n_layers >= 0 && n_loops >= 0 && n_verts >= 0, "negative count");
        require(n_loops <= 0x7fffffffLL && n_verts <= 0x7fffffffLL, "more than 2^31 - 1 items");
        require(layer_loop_off != nullptr && loop_vert_off != nullptr, "offsets are NULL");
        require(n_verts == 0 || xy != nullptr, "xy is NULL");
        require(layer_loop_off[0] == 0 && layer_loop_off[n_layers] == n_loops,
                "layer_loop_off must run from 0 to n_loops");
        for (int32_t l = 0; l < n_layers; ++l)
            require(layer_loop_off[l] <= layer_loop_off[l + 1], "layer_loop_off decreases");
        require(loop_vert_off[0] == 0 && loop_vert_off[n_loops] == n_verts,
                "loop_vert_off must run from 0 to n_verts");
        for (int64_t L = 0; L < n_loops; ++L)
            require(loop_vert_off[L] <= loop_vert_off[L + 1], "loop_vert_off decreases");
        for (int64_t i = 0; i < 2 * n_verts; ++i) require(isfinite(xy[i]), "non-finite vertex");
        if (edge_id)
            for (int64_t i = 0; i < n_verts; ++i) require(edge_id[i] >= 0, "negative edge id");
        cudaStream_t s = (cudaStream_t)stream;
        c = new csl_contours();
        c->n_layers = n_layers;
        c->on_device = 1;
        c->n_loops = n_loops;
        c->n_verts = n_verts;
        auto up = [&](void** dst, const void* src, size_t bytes) {
            if (cudaMalloc(dst, bytes ? bytes : 16) != cudaSuccess) {
                cudaGetLastError();
                fail(CSL_ERR_OOM, "device allocation of the contours failed");
            }
            if (bytes) CSL_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s));
        };
        up((void**)&c->layer_loop_off, layer_loop_off, (size_t)(n_layers + 1) * 8);
        up((void**)&c->loop_vert_off, loop_vert_off, (size_t)(n_loops + 1) * 8);
        up((void**)&c->xy, xy, (size_t)n_verts * 8);
        if (edge_id) up((void**)&c->edge_id, edge_id, (size_t)n_verts * 4);
        CSL_CUDA(cudaStreamSynchronize(s));
        *out = c;
    });
    if (st != CSL_OK && c) csl_contours_free(c);
    return st;
}

csl_status csl_slice_layers(csl_lattice* L, const csl_slice_desc* desc, void* stream,
                            csl_contours** out) {
    return guard([&] {
        require(L != nullptr, "lattice is NULL");
        validate_desc(desc);
        const csl_slice_desc d = *desc;
        const bool want_contours = !(d.flags & CSL_SLICE_NO_CONTOURS);
        require(!want_contours || out != nullptr, "out is NULL");
        if (out) *out = nullptr;
        const bool on_dev = (d.flags & CSL_SLICE_CONTOURS_ON_DEVICE) != 0;
        const bool want_eid = (d.flags & CSL_SLICE_EDGE_IDS) != 0;
        cudaStream_t s = (cudaStream_t)stream;
        SlicePlan p = make_plan(L, d);
        p.fused = wants_fused(d, p);
        // a workspace budget: one chunk in flight, chunks sized from a first
        // chunk's measured workspace, contours to the host chunk by chunk
        const bool budgeted = d.workspace_budget > 0;
        if (budgeted) {
            require_arg(!(d.flags & CSL_SLICE_CONTOURS_ON_DEVICE),
                        "workspace_budget needs host contours");
            require_arg(!L->host_resident, "workspace_budget needs a device-resident lattice");
            require_arg(d.chunk_layers == 0, "workspace_budget sizes the chunks itself");
            require_arg(!(d.flags & CSL_SLICE_TIME_KERNELS), "workspace_budget: no stage timing");
        }
        device_bytes_peak_and_reset();
        const int64_t live_at_start = device_bytes_live();
        launches_and_reset();
        csl_stats st = {};
        st.field_kernel = p.kernel == kFieldFootprint ? CSL_FIELD_FOOTPRINT : CSL_FIELD_BLOCK;
        st.tile = p.T;
        st.slab = p.S;
        st.stage_records = p.K;
        st.fused = p.fused ? 1 : 0;
        const bool time_kernels = (d.flags & CSL_SLICE_TIME_KERNELS) != 0;
        const bool count_pairs = (d.flags & CSL_SLICE_COUNT_PAIRS) != 0;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (time_kernels) {
            CSL_CUDA(cudaEventCreate(&ev0));
            CSL_CUDA(cudaEventCreate(&ev1));
        }
        // times the enqueued work of f() with events on the stream (when asked)
        auto timed = [&](double& acc, const std::function<void()>& f) {
            if (!time_kernels) { f(); return; }
            CSL_CUDA(cudaEventRecord(ev0, s));
            f();
            CSL_CUDA(cudaEventRecord(ev1, s));
            CSL_CUDA(cudaEventSynchronize(ev1));
            float ms = 0.0f;
            CSL_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
            acc += ms;
        };
        DevBuf pair_count;
        if (count_pairs) {
            pair_count.alloc(16, s);
            CSL_CUDA(cudaMemsetAsync(pair_count.get(), 0, 16, s));
        }
        auto finish_stats = [&] {
            if (time_kernels) {
                cudaEventDestroy(ev0);
                cudaEventDestroy(ev1);
            }
            st.device_bytes_peak = device_bytes_peak_and_reset() - live_at_start;
            st.kernel_launches = launches_and_reset();
            t_stats = st;
        };

        const int64_t plane = (int64_t)d.nx * d.ny;
        // with a budget the first chunk is two slabs (a measurement), the
        // others as many whole slabs as fit
        const int chunk0 = budgeted ? std::min(p.chunk, 2 * p.S) : p.chunk;
        const int n_chunks = d.n_layers > 0 ? (int)ceil_div(d.n_layers, chunk0) : 0;
        // Chunks in flight: one, unless the lattice is host-resident. With two,
        // chunk k's window copy, binning and field run on streams[k % 2] with
        // their own Sigma and mask buffers, and every chunk's contour stage runs
        // on one stream of the highest priority once its field is done, so that
        // its kernels are dispatched between the next chunk's field CTAs rather
        // than after all of them, and its size read-backs overlap that field; a
        // chunk's buffers are reused by chunk k + 2 once its contours are done
        // (100M workload, host-resident: 379 -> 333 ms per step with the
        // priority stream and the current field kernel together). For a
        // device-resident lattice one chunk at a time measured faster (100M:
        // 314.4 ms against 332.5 ms with two in flight and the priority stream):
        // the field kernel's CTAs fill the SMs' shared memory, so the contour
        // kernels do not run beside them, and the two compete for L2.
        const int n_par =
            (n_chunks > 1 && !time_kernels && !budgeted && L->host_resident) ? 2 : 1;
        struct Side {
            cudaStream_t s2 = nullptr, cs = nullptr;
            cudaEvent_t fork = nullptr, field_done[2] = {}, cont_done[2] = {};
            ~Side() {
                if (s2) cudaStreamSynchronize(s2);
                if (cs) cudaStreamSynchronize(cs);
                if (fork) cudaEventDestroy(fork);
                for (int b = 0; b < 2; ++b) {
                    if (field_done[b]) cudaEventDestroy(field_done[b]);
                    if (cont_done[b]) cudaEventDestroy(cont_done[b]);
                }
                if (s2) cudaStreamDestroy(s2);
                if (cs) cudaStreamDestroy(cs);
            }
        } side;
        cudaStream_t streams[2] = {s, s};
        if (n_par == 2) {
            int prio_lo = 0, prio_hi = 0;
            CSL_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
            CSL_CUDA(cudaStreamCreateWithFlags(&side.s2, cudaStreamNonBlocking));
            CSL_CUDA(cudaStreamCreateWithPriority(&side.cs, cudaStreamNonBlocking, prio_hi));
            CSL_CUDA(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
            for (int b = 0; b < 2; ++b) {
                CSL_CUDA(cudaEventCreateWithFlags(&side.field_done[b], cudaEventDisableTiming));
                CSL_CUDA(cudaEventCreateWithFlags(&side.cont_done[b], cudaEventDisableTiming));
            }
            CSL_CUDA(cudaEventRecord(side.fork, s));   // both streams follow earlier work on s
            CSL_CUDA(cudaStreamWaitEvent(side.s2, side.fork, 0));
            CSL_CUDA(cudaStreamWaitEvent(side.cs, side.fork, 0));
            streams[1] = side.s2;
        }
        DevBuf sigma_ws[2], mask_ws[2];
        FusedVerts fv_ws[2];
        int chunk_alloc = std::min(chunk0, std::max(d.n_layers, 1));
        const int64_t mask_layer = mask_words_per_layer(d.nx, d.ny);
        const int64_t n_tiles = (int64_t)p.ntx * p.nty;
        // the per-chunk buffers for chunks of up to `layers` layers (grown in place)
        auto chunk_buffers = [&](int layers) {
            chunk_alloc = layers;
            for (int b = 0; b < n_par; ++b) {
                // without contours nothing reads the Sigma plane: the field kernel
                // then writes only the mask (the binary image) unless sigma_out is
                // set; the fused pass leaves vertex lists instead of a plane
                if (!d.sigma_out && want_contours && !p.fused && d.n_layers > 0)
                    sigma_ws[b].ensure((size_t)layers * plane * 4, streams[b]);
                if ((want_contours || d.mask_out) && d.n_layers > 0)
                    mask_ws[b].ensure((size_t)layers * mask_layer * 4, streams[b]);
                if (p.fused && d.n_layers > 0) {
                    FusedVerts& f = fv_ws[b];
                    f.tbase.ensure((size_t)layers * n_tiles * 4, streams[b]);
                    f.roff.ensure((size_t)layers * n_tiles * (p.T + 1) * 2, streams[b]);
                    f.saddle.ensure((size_t)layers * mask_layer * 4, streams[b]);
                    f.counter.ensure(8, streams[b]);
                    // first guess: a crossing per 4 pixel-layers (grown on overflow)
                    int64_t cap = std::max<int64_t>((int64_t)1 << 20, (int64_t)layers * plane / 4);
                    cap = std::min<int64_t>(cap, 0xffffffffLL);
                    if (cap > f.cap) {
                        f.cap = cap;
                        f.verts.ensure((size_t)f.cap * 8, streams[b]);
                    }
                }
            }
        };
        chunk_buffers(chunk_alloc);

        std::vector<ChunkContours> dev_chunks;
        // Host output: the vertices of each chunk are copied to the host while
        // the next chunks are computed (a second stream), into the largest
        // cached page-locked block, as far as it reaches; the rest is copied
        // at the end. Without a cached block everything is copied at the end.
        struct Spec {
            void* block = nullptr;
            size_t bytes = 0, eid_off = 0;
            int64_t cap = 0;          // vertices that fit
            int64_t copied = 0;       // vertices already copied (chunks 0..k)
            cudaStream_t cs = nullptr;
            cudaEvent_t ev = nullptr;
            ~Spec() {
                if (cs) cudaStreamSynchronize(cs);
                if (ev) cudaEventDestroy(ev);
                if (cs) cudaStreamDestroy(cs);
                if (block) host_block_free(block);
            }
        } spec;
        if (want_contours && !on_dev && d.n_layers > 0) {
            spec.block = host_block_take_largest(&spec.bytes);
            if (spec.block) {
                spec.eid_off = vertex_block_eid_offset(spec.bytes, want_eid);
                spec.cap = want_eid ? std::min<int64_t>(spec.eid_off / 8,
                                                        (spec.bytes - spec.eid_off) / 4)
                                    : (int64_t)(spec.bytes / 8);
                // with a budget the copies run on the chunk's stream (its
                // buffers are freed right after, in stream order)
                if (!budgeted) {
                    CSL_CUDA(cudaStreamCreateWithFlags(&spec.cs, cudaStreamNonBlocking));
                    CSL_CUDA(cudaEventCreateWithFlags(&spec.ev, cudaEventDisableTiming));
                }
            }
        }
        bool spec_all = spec.block != nullptr;   // every chunk's vertices went to the block
        // Device contours are assembled in place: every chunk writes its
        // vertices, edge ids and loop offsets into arrays that grow behind
        // fixed address ranges (physical memory mapped as they grow), so no
        // gather copy follows the last chunk and no second copy is held.
        GrowMap gm_xy, gm_eid, gm_loop;
        ChunkDest dest;
        bool in_place = on_dev && want_contours && d.n_layers > 0 && growmap_available();
        if (in_place) {
            size_t free_b = 0, total_b = 0;
            CSL_CUDA(cudaMemGetInfo(&free_b, &total_b));
            gm_xy.reserve(total_b);
            if (want_eid) gm_eid.reserve(total_b / 2);
            gm_loop.reserve(total_b);
            dest.xy = static_cast<float2*>(gm_xy.base());
            dest.eid = want_eid ? static_cast<int32_t*>(gm_eid.base()) : nullptr;
            dest.loop_off = static_cast<int64_t*>(gm_loop.base());
            dest.make_room = [&](int64_t verts, int64_t loop_entries) {
                gm_xy.ensure((size_t)verts * 8);
                if (want_eid) gm_eid.ensure((size_t)verts * 4);
                gm_loop.ensure((size_t)loop_entries * 8);
            };
        }
        auto contour_stage = [&](int k, const ChunkGeom& g) {
            cudaStream_t ks = streams[k % n_par];
            if (n_par == 2) {   // the contour stream, after this chunk's field
                ks = side.cs;
                CSL_CUDA(cudaStreamWaitEvent(ks, side.field_done[k % 2], 0));
            }
            const float* sigma = d.sigma_out ? d.sigma_out + (int64_t)g.first_layer * plane
                                             : sigma_ws[k % n_par].as<float>();   // null: fused
            ChunkContours cc;
            cc.n_layers = g.n_layers;
            timed(st.contour_ms, [&] {
                contours_chunk(g, L->C, sigma, mask_ws[k % n_par].as<uint32_t>(), want_eid, cc,
                               ks, nullptr, p.fused ? &fv_ws[k % n_par] : nullptr,
                               in_place ? &dest : nullptr);
            });
            if (n_par == 2) CSL_CUDA(cudaEventRecord(side.cont_done[k % 2], ks));
            st.crossings += cc.n_verts;
            st.loops += cc.n_loops;
            dest.v_base += cc.n_verts;
            dest.l_base += cc.n_loops;
            if (budgeted) {   // to_host() copies this chunk
            } else if (spec_all && spec.copied + cc.n_verts <= spec.cap) {
                if (cc.n_verts) {
                    CSL_CUDA(cudaEventRecord(spec.ev, ks));
                    CSL_CUDA(cudaStreamWaitEvent(spec.cs, spec.ev, 0));
                    char* base = static_cast<char*>(spec.block);
                    CSL_CUDA(cudaMemcpyAsync(base + spec.copied * 8, cc.xy.get(), cc.n_verts * 8,
                                             cudaMemcpyDeviceToHost, spec.cs));
                    if (want_eid)
                        CSL_CUDA(cudaMemcpyAsync(base + spec.eid_off + spec.copied * 4,
                                                 cc.eid.get(), cc.n_verts * 4,
                                                 cudaMemcpyDeviceToHost, spec.cs));
                }
                spec.copied += cc.n_verts;
            } else {
                spec_all = false;
            }
            dev_chunks.push_back(std::move(cc));
        };
        // A host-resident lattice: each chunk's z window of the sorted records
        // (every record the chunk's slabs can select, with slack) is copied to
        // one of two device windows, and the binner and field kernel see a view
        // of the lattice made of that window.
        std::vector<std::pair<int64_t, int64_t>> wins;
        DevBuf w_rec[2], w_bxy[2], w_zlo[2], w_zhi[2];
        if (L->host_resident) {
            int64_t max_w = 1;
            for (int k = 0; k < n_chunks; ++k) {
                const int first = k * p.chunk;
                const int n = std::min(p.chunk, d.n_layers - first);
                const ChunkGeom g = chunk_geom(L, d, p, first, n);
                const double zf = g.z0 + (double)g.first_layer * g.dz;
                const double zl = g.z0 + (double)(g.first_layer + g.n_layers - 1) * g.dz;
                const double lo_key = zf - g.margin_z - L->max_dz - 2e-3 * (1.0 + fabs(zf)) - fabs(g.dz);
                const double hi_key = zl + g.margin_z + 2e-3 * (1.0 + fabs(zl)) + fabs(g.dz);
                const float* z = L->h_zlo;
                const int64_t a = std::lower_bound(z, z + L->n_edges, lo_key,
                                                   [](float v, double key) { return (double)v < key; }) - z;
                const int64_t b = std::upper_bound(z + a, z + L->n_edges, hi_key,
                                                   [](double key, float v) { return key < (double)v; }) - z;
                wins.emplace_back(a, b);
                max_w = std::max<int64_t>(max_w, b - a);
            }
            for (int b = 0; b < n_par; ++b) {
                w_rec[b].alloc((size_t)max_w * sizeof(csl_rec), streams[b]);
                w_bxy[b].alloc((size_t)max_w * 16, streams[b]);
                w_zlo[b].alloc((size_t)max_w * 4, streams[b]);
                w_zhi[b].alloc((size_t)max_w * 4, streams[b]);
            }
        }
        int prev = -1;
        ChunkGeom g_prev{};
        // a budget: chunks' contours copied to host memory as they finish; the
        // vertices into the cached page-locked block while they fit (at the
        // link's speed, in stream order before the chunk's buffers are
        // freed), else into pageable memory
        struct HostChunk {
            int n = 0;
            int64_t n_loops = 0, n_verts = 0;
            int64_t block_at = -1;   // first vertex in spec.block, or -1
            std::vector<int64_t> layer_loops, loop_off;
            std::vector<float> xy;
            std::vector<int32_t> eid;
        };
        std::vector<HostChunk> host_chunks;
        auto to_host = [&](cudaStream_t ks) {
            ChunkContours& cc = dev_chunks.back();
            HostChunk h;
            h.n = cc.n_layers;
            h.n_loops = cc.n_loops;
            h.n_verts = cc.n_verts;
            h.layer_loops.resize((size_t)h.n + 1);
            h.loop_off.resize((size_t)h.n_loops + 1);
            if (spec_all && spec.copied + h.n_verts <= spec.cap) {
                char* base = static_cast<char*>(spec.block);
                if (h.n_verts) {
                    CSL_CUDA(cudaMemcpyAsync(base + spec.copied * 8, cc.xy.get(), h.n_verts * 8,
                                             cudaMemcpyDeviceToHost, ks));
                    if (want_eid)
                        CSL_CUDA(cudaMemcpyAsync(base + spec.eid_off + spec.copied * 4,
                                                 cc.eid.get(), h.n_verts * 4,
                                                 cudaMemcpyDeviceToHost, ks));
                }
                h.block_at = spec.copied;
                spec.copied += h.n_verts;
            } else {
                spec_all = false;
                h.xy.resize((size_t)h.n_verts * 2);
                if (h.n_verts) read_to_host(h.xy.data(), cc.xy.get(), h.n_verts * 8, ks);
                if (want_eid && h.n_verts) {
                    h.eid.resize((size_t)h.n_verts);
                    read_to_host(h.eid.data(), cc.eid.get(), h.n_verts * 4, ks);
                }
            }
            read_to_host(h.layer_loops.data(), cc.layer_loops.get(), (h.n + 1) * 8, ks);
            read_to_host(h.loop_off.data(), cc.loop_off.get(), (h.n_loops + 1) * 8, ks);
            host_chunks.push_back(std::move(h));
            dev_chunks.pop_back();   // the device copies are freed here
        };
        // on an early exit (an error) no buffer above is freed while the other
        // streams may still use it
        struct Join {
            const Side& sd;
            ~Join() {
                if (sd.s2) cudaStreamSynchronize(sd.s2);
                if (sd.cs) cudaStreamSynchronize(sd.cs);
            }
        } join{side};
        int cur_chunk = chunk0;
        int first = 0;
        for (int k = 0; first < d.n_layers; ++k) {
            const int n = std::min(cur_chunk, d.n_layers - first);
            ChunkGeom g = chunk_geom(L, d, p, first, n);
            cudaStream_t ks = streams[k % n_par];
            csl_lattice view;              // the window of a host-resident lattice
            const csl_lattice* LB = L;     // what the binner and field kernel see
            if (L->host_resident) {
                const int64_t a = wins[k].first, nw = wins[k].second - wins[k].first;
                const int b = k % n_par;
                if (nw > 0) {
                    CSL_CUDA(cudaMemcpyAsync(w_rec[b].get(), L->h_rec + a, (size_t)nw * sizeof(csl_rec),
                                             cudaMemcpyHostToDevice, ks));
                    CSL_CUDA(cudaMemcpyAsync(w_bxy[b].get(), L->h_bxy + a, (size_t)nw * 16,
                                             cudaMemcpyHostToDevice, ks));
                    CSL_CUDA(cudaMemcpyAsync(w_zlo[b].get(), L->h_zlo + a, (size_t)nw * 4,
                                             cudaMemcpyHostToDevice, ks));
                    CSL_CUDA(cudaMemcpyAsync(w_zhi[b].get(), L->h_zhi + a, (size_t)nw * 4,
                                             cudaMemcpyHostToDevice, ks));
                }
                view.n_nodes = L->n_nodes;
                view.n_edges = nw;
                view.R = L->R;
                view.C = L->C;
                view.mode = L->mode;
                for (int c3 = 0; c3 < 3; ++c3) {
                    view.bbox_lo[c3] = L->bbox_lo[c3];
                    view.bbox_hi[c3] = L->bbox_hi[c3];
                }
                view.max_dz = L->max_dz;
                view.max_radius = L->max_radius;
                view.rec.view(w_rec[b].get(), w_rec[b].size());
                view.bxy.view(w_bxy[b].get(), w_bxy[b].size());
                view.zlo.view(w_zlo[b].get(), w_zlo[b].size());
                view.zhi.view(w_zhi[b].get(), w_zhi[b].size());
                view.status.view(L->status.get(), 4);
                LB = &view;
            }
            float* sigma = d.sigma_out ? d.sigma_out + (int64_t)first * plane
                                       : sigma_ws[k % n_par].as<float>();   // null: mask only
            {
                SlabBins bins;
                timed(st.bin_ms, [&] { bin_chunk(LB, g, bins, ks); });
                st.candidate_pairs += bins.n_pairs;
                st.window_records += bins.n_cand;
                uint32_t* mask = (want_contours || d.mask_out) ? mask_ws[k % n_par].as<uint32_t>()
                                                               : nullptr;
                FusedVerts* fv = p.fused ? &fv_ws[k % n_par] : nullptr;
                // chunk k - 2's contours read these buffers
                if (n_par == 2 && k >= 2)
                    CSL_CUDA(cudaStreamWaitEvent(ks, side.cont_done[k % 2], 0));
                auto run_field = [&] {
                    if (mask) CSL_CUDA(cudaMemsetAsync(mask, 0, (size_t)n * mask_layer * 4, ks));
                    if (fv) {
                        CSL_CUDA(cudaMemsetAsync(fv->saddle.get(), 0, (size_t)n * mask_layer * 4, ks));
                        CSL_CUDA(cudaMemsetAsync(fv->counter.get(), 0, 8, ks));
                    }
                    timed(st.field_ms, [&] {
                        field_chunk(LB, g, bins, (float)L->C, sigma, mask,
                                    count_pairs ? pair_count.as<unsigned long long>() : nullptr, ks,
                                    fv);
                    });
                };
                run_field();
                if (fv) {
                    // the vertex lists' capacity was a guess: on overflow, grow it
                    // to what the chunk needs and run the field again
                    uint32_t cnt[2];
                    read_to_host(cnt, fv->counter.get(), 8, ks);
                    if (cnt[1]) {
                        if (count_pairs) fail(CSL_ERR_CAPACITY, "fused vertex lists overflowed "
                                                                "while counting pairs");
                        fv->cap = std::min<int64_t>((int64_t)cnt[0] + cnt[0] / 4 + (1 << 20),
                                                    0xffffffffLL);
                        fv->verts.release();
                        fv->verts.alloc((size_t)fv->cap * 8, ks);
                        run_field();
                        read_to_host(cnt, fv->counter.get(), 8, ks);
                        if (cnt[1]) fail(CSL_ERR_CAPACITY, "fused vertex lists overflowed twice");
                    }
                }
                ++st.field_launches;
                if (d.mask_out) {
                    const int64_t wpr = ceil_div(d.nx, 32);
                    const int64_t n_out = (int64_t)n * d.ny * wpr;
                    k_unpad_mask<<<grid_for(n_out, 256), 256, 0, ks>>>(
                        mask, d.nx, d.ny, n, mask_words_per_row(d.nx), mask_layer,
                        d.mask_out + (int64_t)first * d.ny * wpr);
                    CSL_LAUNCH_CHECK("mask out");
                }
            }
            if (n_par == 2) CSL_CUDA(cudaEventRecord(side.field_done[k % 2], ks));
            ++st.chunks;
            first += n;
            if (n_par == 1) {   // one set of buffers: this chunk's contours now
                if (want_contours) contour_stage(k, g);
                if (budgeted) {
                    if (want_contours) to_host(ks);
                    if (k == 0 && first < d.n_layers) {
                        // the first chunk's workspace per layer sizes the others
                        CSL_CUDA(cudaStreamSynchronize(ks));
                        const int64_t w0 = device_bytes_peak() - live_at_start;
                        if (w0 > d.workspace_budget)
                            fail(CSL_ERR_CAPACITY,
                                 "workspace_budget: a chunk of " + std::to_string(n) +
                                     " layers needs " + std::to_string(w0) + " bytes");
                        const double per_layer = (double)w0 / n;
                        int c = (int)std::min<double>(0.9 * (double)d.workspace_budget / per_layer,
                                                      1e9);
                        // marching squares needs < 2^27 edge words per chunk
                        const int64_t cap = (((int64_t)1 << 27) - 1) / (2 * mask_layer);
                        c = (int)std::min<int64_t>(c, cap);
                        c -= c % p.S;
                        cur_chunk = std::max(c, p.S);
                        if (cur_chunk > chunk_alloc) chunk_buffers(cur_chunk);
                    }
                }
                continue;
            }
            // the previous chunk's contours, while this chunk's field runs
            if (want_contours && prev >= 0) contour_stage(prev, g_prev);
            prev = k;
            g_prev = g;
        }
        if (want_contours && prev >= 0) contour_stage(prev, g_prev);
        if (side.s2) CSL_CUDA(cudaStreamSynchronize(side.s2));
        if (side.cs) CSL_CUDA(cudaStreamSynchronize(side.cs));
        CSL_CUDA(cudaStreamSynchronize(s));
        check_lattice_status(L, s);
        if (count_pairs) {
            int64_t pc[2];
            read_to_host(pc, pair_count.get(), 16, s);
            st.contributing_pairs = pc[0];
            st.evaluated_terms = pc[1];
        }
        if (!want_contours) {
            finish_stats();
            return;
        }

        if (budgeted) {   // assemble the host chunks
            int64_t n_loops = 0, n_verts = 0;
            for (auto& h : host_chunks) { n_loops += h.n_loops; n_verts += h.n_verts; }
            csl_contours* c = nullptr;
            if (spec_all) {   // every chunk's vertices are in the block already
                c = new_host_contours(d.n_layers, n_loops, n_verts, want_eid, spec.block);
                spec.block = nullptr;   // now owned by c
            } else {
                c = new_host_contours(d.n_layers, n_loops, n_verts, want_eid);
            }
            const char* blk = static_cast<const char*>(spec.block);
            int64_t lb = 0, vb = 0;
            int layer = 0;
            c->layer_loop_off[0] = 0;
            c->loop_vert_off[0] = 0;
            for (auto& h : host_chunks) {
                for (int i = 1; i <= h.n; ++i) c->layer_loop_off[layer + i] = h.layer_loops[i] + lb;
                for (int64_t i = 1; i <= h.n_loops; ++i) c->loop_vert_off[lb + i] = h.loop_off[i] + vb;
                if (h.block_at < 0) {
                    if (h.n_verts) memcpy(c->xy + 2 * vb, h.xy.data(), (size_t)h.n_verts * 8);
                    if (want_eid && h.n_verts)
                        memcpy(c->edge_id + vb, h.eid.data(), (size_t)h.n_verts * 4);
                } else if (blk && h.n_verts) {   // in the block, but the result is elsewhere
                    memcpy(c->xy + 2 * vb, blk + h.block_at * 8, (size_t)h.n_verts * 8);
                    if (want_eid)
                        memcpy(c->edge_id + vb, blk + spec.eid_off + h.block_at * 4,
                               (size_t)h.n_verts * 4);
                }
                lb += h.n_loops;
                vb += h.n_verts;
                layer += h.n;
            }
            finish_stats();
            *out = c;
            return;
        }
        // Gather the chunks into the result: offsets are rebased on the device,
        // then every array is copied straight to its place (device or host).
        int64_t n_loops = 0, n_verts = 0;
        for (auto& cc : dev_chunks) { n_loops += cc.n_loops; n_verts += cc.n_verts; }
        csl_contours* c = nullptr;
        if (in_place) {   // the arrays are complete: hand them over, offsets per layer only
            c = new csl_contours();
            memset(c, 0, sizeof(*c));
            c->n_layers = d.n_layers;
            c->on_device = 1;
            c->n_loops = n_loops;
            c->n_verts = n_verts;
            if (cudaMalloc((void**)&c->layer_loop_off, (size_t)(d.n_layers + 1) * 8) != cudaSuccess) {
                cudaGetLastError();
                delete c;
                fail(CSL_ERR_OOM, "device allocation of the contours failed");
            }
            int layer = 0;
            for (auto& cc : dev_chunks) {   // rebased already; entry 0 repeats the last end
                CSL_CUDA(cudaMemcpyAsync(c->layer_loop_off + layer, cc.layer_loops.get(),
                                         (size_t)(cc.n_layers + 1) * 8, cudaMemcpyDeviceToDevice, s));
                layer += cc.n_layers;
            }
            CSL_CUDA(cudaStreamSynchronize(s));
            c->xy = static_cast<float*>(gm_xy.hand_over());
            c->edge_id = want_eid ? static_cast<int32_t*>(gm_eid.hand_over()) : nullptr;
            c->loop_vert_off = static_cast<int64_t*>(gm_loop.hand_over());
            dev_chunks.clear();
            finish_stats();
            *out = c;
            return;
        }
        if (on_dev) {
            c = new csl_contours();
            memset(c, 0, sizeof(*c));
            c->n_layers = d.n_layers;
            c->on_device = 1;
            c->n_loops = n_loops;
            c->n_verts = n_verts;
            auto dst_alloc = [&](void** p, size_t b) {
                if (cudaMalloc(p, b ? b : 16) != cudaSuccess) {
                    cudaGetLastError();
                    csl_contours_free(c);
                    fail(CSL_ERR_OOM, "device allocation of the contours failed");
                }
            };
            dst_alloc((void**)&c->layer_loop_off, (size_t)(d.n_layers + 1) * 8);
            dst_alloc((void**)&c->loop_vert_off, (size_t)(n_loops + 1) * 8);
            dst_alloc((void**)&c->xy, (size_t)n_verts * 8);
            if (want_eid) dst_alloc((void**)&c->edge_id, (size_t)n_verts * 4);
        } else if (spec_all) {
            c = new_host_contours(d.n_layers, n_loops, n_verts, want_eid, spec.block);
            spec.block = nullptr;   // now owned by c
        } else {
            c = new_host_contours(d.n_layers, n_loops, n_verts, want_eid);
        }
        const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        timed(st.output_ms, [&] {
            int64_t lb = 0, vb = 0;
            int layer = 0;
            for (auto& cc : dev_chunks) {
                const int n = cc.n_layers;
                if (lb) {
                    k_add_i64<<<grid_for(n + 1, 256), 256, 0, s>>>(cc.layer_loops.as<int64_t>(),
                                                                   n + 1, lb);
                    CSL_LAUNCH_CHECK("rebase layer offsets");
                }
                if (vb) {
                    k_add_i64<<<grid_for(cc.n_loops + 1, 256), 256, 0, s>>>(
                        cc.loop_off.as<int64_t>(), cc.n_loops + 1, vb);
                    CSL_LAUNCH_CHECK("rebase loop offsets");
                }
                // entry 0 of each chunk duplicates the previous chunk's last entry
                CSL_CUDA(cudaMemcpyAsync(c->layer_loop_off + layer, cc.layer_loops.get(),
                                         (size_t)(n + 1) * 8, kind, s));
                CSL_CUDA(cudaMemcpyAsync(c->loop_vert_off + lb, cc.loop_off.get(),
                                         (size_t)(cc.n_loops + 1) * 8, kind, s));
                if (cc.n_verts && !(spec_all && !on_dev)) {   // else already on the host
                    CSL_CUDA(cudaMemcpyAsync(c->xy + 2 * vb, cc.xy.get(), cc.n_verts * 8, kind, s));
                    if (want_eid)
                        CSL_CUDA(cudaMemcpyAsync(c->edge_id + vb, cc.eid.get(), cc.n_verts * 4,
                                                 kind, s));
                }
                lb += cc.n_loops;
                vb += cc.n_verts;
                layer += n;
            }
            if (d.n_layers == 0) {
                const int64_t zero = 0;
                CSL_CUDA(cudaMemcpyAsync(c->layer_loop_off, &zero, 8,
                                         on_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
                CSL_CUDA(cudaMemcpyAsync(c->loop_vert_off, &zero, 8,
                                         on_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
            }
            CSL_CUDA(cudaStreamSynchronize(s));
            if (spec.cs) CSL_CUDA(cudaStreamSynchronize(spec.cs));
        });
        dev_chunks.clear();
        finish_stats();
        *out = c;
    });
}

csl_status csl_volume_fraction(csl_lattice* L, const csl_cells* cells, float* vf_out,
                               void* stream) {
    return guard([&] {
        require(L != nullptr, "lattice is NULL");
        require_device_resident(L);
        validate_cells_or_fail(cells);
        require(vf_out != nullptr, "vf_out is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        launches_and_reset();
        vf_forward(L, *cells, vf_out, s);
        CSL_CUDA(cudaStreamSynchronize(s));
        check_lattice_status(L, s);
        t_stats = csl_stats{};
        t_stats.kernel_launches = launches_and_reset();
    });
}

csl_status csl_volume_fraction_backward(csl_lattice* L, const csl_cells* cells,
                                        const float* grad_vf, float* grad_radius,
                                        float* grad_nodes, void* stream) {
    return guard([&] {
        require(L != nullptr, "lattice is NULL");
        require_device_resident(L);
        validate_cells_or_fail(cells);
        require(grad_vf != nullptr, "grad_vf is NULL");
        require(L->n_edges == 0 || grad_radius != nullptr, "grad_radius is NULL");
        require(L->n_nodes == 0 || grad_nodes != nullptr, "grad_nodes is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        launches_and_reset();
        vf_backward(L, *cells, grad_vf, grad_radius, grad_nodes, s);
        CSL_CUDA(cudaStreamSynchronize(s));
        t_stats = csl_stats{};
        t_stats.kernel_launches = launches_and_reset();
    });
}

csl_status csl_debug_slab_bins(csl_lattice* L, const csl_slice_desc* desc, int32_t first_layer,
                               int32_t n_slab_layers, int64_t* tile_off, int32_t* ids,
                               int64_t capacity, int64_t* n_ids, void* stream) {
    return guard([&] {
        require(L != nullptr && tile_off != nullptr && n_ids != nullptr, "NULL argument");
        require_device_resident(L);
        validate_desc(desc);
        require(n_slab_layers >= 1 && first_layer >= 0, "bad slab");
        cudaStream_t s = (cudaStream_t)stream;
        csl_slice_desc d = *desc;
        if (d.n_layers < first_layer + n_slab_layers) d.n_layers = first_layer + n_slab_layers;
        SlicePlan p = make_plan(L, d);
        p.fused = wants_fused(d, p);   // the bins of the pass csl_slice_layers would run
        ChunkGeom g = chunk_geom(L, d, p, first_layer, n_slab_layers);
        g.S = n_slab_layers;
        g.n_slabs = 1;
        SlabBins bins;
        bin_chunk(L, g, bins, s);
        const int n_tiles = g.ntx * g.nty;
        std::vector<uint32_t> ts(n_tiles), te(n_tiles), vals(bins.n_pairs), sid(L->n_edges);
        read_to_host(ts.data(), bins.tile_start.get(), n_tiles * 4, s);
        read_to_host(te.data(), bins.tile_end.get(), n_tiles * 4, s);
        if (bins.n_pairs) read_to_host(vals.data(), bins.vals.get(), bins.n_pairs * 4, s);
        if (L->n_edges) read_to_host(sid.data(), L->sid.get(), L->n_edges * 4, s);
        *n_ids = bins.n_pairs;
        tile_off[0] = 0;
        int64_t pos = 0;
        for (int t = 0; t < n_tiles; ++t) {
            std::vector<int32_t> list;
            for (uint32_t i = ts[t]; i < te[t]; ++i) list.push_back((int32_t)(sid[vals[i]] & 0x7fffffffu));
            std::sort(list.begin(), list.end());
            if (ids && pos + (int64_t)list.size() <= capacity)
                memcpy(ids + pos, list.data(), list.size() * 4);
            pos += (int64_t)list.size();
            tile_off[t + 1] = pos;
        }
        if (pos > capacity) fail(CSL_ERR_CAPACITY, "ids capacity too small");
    });
}

}  // extern "C"
