// Internal interfaces of the slicing pipeline (binner, field, contours).
#pragma once

#include <functional>
#include <vector>

#include "lattice.cuh"

namespace csl {

constexpr int kTile = 16;        // pixels per tile side of the block field kernel
constexpr int kFieldThreads = 256;

// Field kernels: the pixel-block kernel (field.cu: warps own 8 x 4-pixel
// blocks of a 16 x 16 tile, sums in registers) and the footprint kernel
// (field_fp.cu: a warp per layer walks each edge's footprint, sums in shared
// memory; tiles of 16 or 32 pixels).
enum FieldKernel : int32_t { kFieldBlock = 1, kFieldFootprint = 2 };

// Geometry of one streamed chunk of layers.
struct ChunkGeom {
    // grid
    int32_t nx, ny, ntx, nty;
    double x0, y0, px, z0, dz;
    // chunk: layers [first_layer, first_layer + n_layers), slabs of S layers
    int32_t first_layer, n_layers, S, n_slabs;
    // lattice
    double R;
    float margin_xy;   // xy expansion of a clipped edge's box (R plus rounding slack)
    float margin_z;    // z expansion (R plus rounding slack)
    // tile side in pixels, field kernel, records per staged copy (footprint kernel)
    int32_t T = kTile;
    int32_t kernel = kFieldBlock;
    int32_t K = 256;
    // fused field and contour pass: tiles also take their next column and row
    // (binner halo), and the field kernel leaves vertex lists instead of Sigma
    bool fused = false;
};

// Per-slab binning results (device).
struct SlabBins {
    DevBuf keys, vals;          // sorted pairs: key = slab * n_tiles + tile, val = record position
    DevBuf recs;                // csl_rec per entry, in entry order: each tile's list contiguous
    DevBuf tile_start, tile_end;// uint32 [n_slabs * n_tiles]
    int64_t n_pairs = 0;
    int64_t n_cand = 0;         // records examined: the slabs' z windows, summed
};

// Sizes that a chunk's pipeline discovers on the host (each needs a read
// back). A planning run records them; a replay run uses them instead, reads
// nothing back (so it can be captured in a CUDA graph), bounds every write by
// them and sets *flag when the device finds other sizes (the inputs changed).
struct ChunkPlan {
    int64_t n_cand = 0, max_window = 0, n_pairs = 0;     // binner
    int64_t n_cross = 0, ns = 0, nl = 0, n_loops = 0;    // contours
};
struct Replay {
    bool replay = false;         // false: record into *plan; true: use *plan
    ChunkPlan* plan = nullptr;
    uint32_t* flag = nullptr;    // device word, OR-ed with 1 on a size mismatch
};

// Bins the lattice's records into (slab, tile) lists for one chunk.
void bin_chunk(const csl_lattice* L, const ChunkGeom& g, SlabBins& out, cudaStream_t s,
               const Replay* rp = nullptr);

// Inside mask of a chunk (the binary image of Sec. 4): bit I % 32 of word
// [layer][J][I / 32] is set when padded sample (I, J), i.e. pixel (I-1, J-1),
// has Sigma >= C. Rows J in [0, ny + 2); the padding ring stays 0.
inline int64_t mask_words_per_row(int nx) { return ceil_div((int64_t)nx + 2, 32); }
inline int64_t mask_words_per_layer(int nx, int ny) {
    return mask_words_per_row(nx) * ((int64_t)ny + 2);
}

// Output of the fused field and contour pass (field_fp.cu) in place of a Sigma
// plane. A tile owns the padded samples of its pixels (and, in the first tile
// column / row, the padding column / row before them) and the grid edges from
// them to the next sample in x and in y. For every (layer, tile) its crossing
// vertices are listed in edge-id order (rows, then samples, the x edge before
// the y edge) at verts[tbase[layer][tile] + roff[layer][tile][row + 1] + rank
// in the row], row in [-1, T - 1] tile-local; `saddle` has the mask's layout,
// bit (I, J) set when cell (I, J) is a saddle whose inside corners join (mean
// of the four corners >= C). Vertices are the same float expressions as the
// unfused contour stage evaluates from Sigma, so both give identical contours.
struct FusedVerts {
    DevBuf tbase;     // uint32 [n_layers][n_tiles]
    DevBuf roff;      // uint16 [n_layers][n_tiles][T + 1]
    DevBuf verts;     // float2 [cap]
    DevBuf saddle;    // uint32 [n_layers][mask words per layer]
    DevBuf counter;   // uint32 [2]: vertices allocated (even past cap), overflow flag
    int64_t cap = 0;
};

// Sigma for every pixel of the chunk's layers: sigma[layer][ny][nx], and the
// inside mask (OR-ed into `mask`, which must be zero on entry; may be null).
// count_pairs (device, may be null): [0] += the number of (pixel, layer, edge)
// terms that are nonzero, [1] += the number of terms evaluated.
// With g.fused, fv (allocated for the chunk, saddle and counter zero) receives
// the vertex lists and sigma may be null.
void field_chunk(const csl_lattice* L, const ChunkGeom& g, const SlabBins& bins, float C,
                 float* sigma, uint32_t* mask, unsigned long long* count_pairs, cudaStream_t s,
                 FusedVerts* fv = nullptr);
// The footprint kernel's launch (field_fp.cu); org: the chunk's origin tables.
void field_chunk_fp(const ChunkGeom& g, const SlabBins& bins, float C, const float2* org,
                    uint32_t* err, float* sigma, uint32_t* mask, unsigned long long* count_pairs,
                    cudaStream_t s, FusedVerts* fv);

// Field of many chunks (the jobs of a batch, one chunk each) in one
// persistent launch: CTAs take (job, slab, tile) items from a queue sorted
// longest tile list first. Every job has the same slab depth.
struct FieldBatchJob {
    const csl_lattice* L;
    ChunkGeom g;
    const SlabBins* bins;   // must stay allocated (same buffers) while the batch lives
    float* sigma;
    uint32_t* mask;         // zero on entry of every run
    uint32_t* err;          // device word OR-ed with ST_TIMEOUT when a wait gives up
};
struct FieldBatch {
    DevBuf jobs, fp_jobs, origins, items, keys, vals, tmp_keys, tmp_vals, counter;
    int64_t n_items = 0;
    int S = 0;
    int kernel = kFieldBlock, T = kTile, K = 256;   // the jobs' field kernel, tile, staging chunk
};
// One-time tables (synchronises s).
void field_batch_prepare(const std::vector<FieldBatchJob>& jobs, FieldBatch& fb, cudaStream_t s);
// The footprint kernel's part of them (field_fp.cu): the jobs as the persistent
// footprint kernel reads them (host bytes, one record per job), and its launch.
void fp_batch_jobs(const std::vector<FieldBatchJob>& jobs, const float2* const* orgs,
                   std::vector<unsigned char>& host);
void fp_batch_launch(const void* jobs, const uint2* items, const uint32_t* order, uint32_t n,
                     uint32_t* counter, int T, int S, int K, int n_ctas, cudaStream_t s);
// The run itself: queue order, counter reset, persistent launch of n_ctas
// CTAs; reads nothing back (capturable in a CUDA graph).
void field_batch_run(FieldBatch& fb, int n_ctas, cudaStream_t s);

// Contours of the chunk's layers (device arrays, layer-local edge ids).
struct ChunkContours {
    int64_t n_verts = 0, n_loops = 0;
    int32_t n_layers = 0;   // layers of the chunk (set by the slicing driver)
    DevBuf layer_loops;   // int64 [n_layers + 1] loop offsets per layer (chunk-local)
    DevBuf loop_off;      // int64 [n_loops + 1] vertex offsets (chunk-local)
    DevBuf xy;            // float2 [n_verts]
    DevBuf eid;           // int32 [n_verts]
};
// A result assembled in place (device contours of a whole slice): a chunk
// writes its vertices from v_base and its loop offsets from l_base of these
// arrays, with the bases added to the offsets (and its layer_loops rebased by
// l_base), after make_room(vertices, loop entries) has made the arrays reach
// v_base + its vertices and l_base + its loops + 1.
struct ChunkDest {
    float2* xy = nullptr;
    int32_t* eid = nullptr;       // when edge ids are wanted
    int64_t* loop_off = nullptr;
    int64_t v_base = 0, l_base = 0;
    std::function<void(int64_t, int64_t)> make_room;
};

// Contours of a chunk. In a replay (rp->replay), out's arrays must already
// hold rp->plan's sizes; they are filled in place.
// With fv (the fused pass's vertex lists) sigma is not read and may be null.
// With dest, out keeps only layer_loops (rebased) and the counts.
void contours_chunk(const ChunkGeom& g, double C, const float* sigma, const uint32_t* mask,
                    bool want_eid, ChunkContours& out, cudaStream_t s, const Replay* rp = nullptr,
                    const FusedVerts* fv = nullptr, const ChunkDest* dest = nullptr);

// Slicing request resolution (api.cu): tile / slab / chunk sizes and the
// binner's rounding margin; the geometry of one chunk; argument checks that
// fail with CSL_ERR_INVALID_ARG.
struct SlicePlan {
    int S, chunk, ntx, nty;
    float margin;
    int T, kernel, K;
    bool fused = false;   // the fused field and contour pass (set by the slicing call)
};
// Whether a slicing request runs the fused pass: the footprint kernel, contours
// wanted, and CSL_SLICE_FUSED.
bool wants_fused(const csl_slice_desc& d, const SlicePlan& p);
SlicePlan make_plan(const csl_lattice* L, const csl_slice_desc& d);
ChunkGeom chunk_geom(const csl_lattice* L, const csl_slice_desc& d, const SlicePlan& p, int first,
                     int n);
void validate_desc(const csl_slice_desc* d);
void require_arg(bool ok, const char* msg);
// Fails with NOT_READY for a host-resident lattice (slicing is its only use).
void require_device_resident(const csl_lattice* L);

// Reads and clears the lattice's device status word; CSL_ERR_TIMEOUT when a
// device wait of an earlier kernel gave up (synchronises s).
void check_lattice_status(const csl_lattice* L, cudaStream_t s);

// Volume fraction per density cell and its adjoint (vf.cu).
void vf_forward(const csl_lattice* L, const csl_cells& cells, float* vf, cudaStream_t s);
void vf_backward(csl_lattice* L, const csl_cells& cells, const float* grad_vf, float* grad_radius,
                 float* grad_nodes, cudaStream_t s);
void validate_cells_or_fail(const csl_cells* c);

}  // namespace csl
