/*
 * cslice: slicing of convolution-surface lattices on one GPU (sm_103a).
 *
 * C ABI of libcslice.so. Plain pointers and sizes only; nothing throws across
 * this boundary. Every call returns a csl_status; on failure
 * csl_last_error() returns a message for the calling thread.
 *
 * The method (arxiv 2101.05031):
 *   - lattice: graph of nodes v_i (float3) and edges e_j = (v_s, v_e, r_j)
 *     (Sec. 3.1);
 *   - field:  Sigma(p) = sum_j w_j * int_{e_j} f(p - x) de with the quartic
 *     compact kernel f = (1 - |p - x|^2 / R^2)^2 inside radius R (Eq. 5, 6),
 *     evaluated per edge in closed form (Eq. 7, arc-length measure);
 *   - solid:  p is inside iff Sigma(p) >= C (the paper's F = -C + Sigma, with
 *     its sign read so that the skeleton is inside);
 *   - slicing: planes z_k = z0 + k dz, only edges whose swept sphere meets the
 *     plane contribute (Eq. 8, Sec. 4 Steps 1-6); the binary image is traced by
 *     marching squares into closed contours (Sec. 4, last paragraph);
 *   - density: per-cell volume fraction of the solid (Eq. 9), here smoothed by
 *     a sigmoid so that it can be differentiated for radius tuning (Sec. 5.4).
 *
 * Weight of an edge (csl_params.mode):
 *   CSL_MODE_PHYSICAL  radius[j] is the physical strut radius rho_j and
 *                      w_j = C * 15 R^4 / (16 (R^2 - rho_j^2)^(5/2)), which
 *                      puts the iso-surface of an isolated long strut at
 *                      distance rho_j; requires 0 < rho_j < R.
 *   CSL_MODE_RAW       w_j = radius[j], the paper's r_i taken literally.
 *
 * Streams: every call enqueues its GPU work on the caller's CUDA stream
 * (a cudaStream_t passed as void*; NULL = legacy default stream). Calls that
 * return host data synchronise that stream before returning.
 * Memory: the library allocates its own device memory with the stream-ordered
 * allocator (cudaMallocAsync) on that stream and frees it the same way; what
 * outlives the call (a lattice, a batch) comes from the same pool on the
 * legacy default stream, synchronised, and is freed after a device
 * synchronisation. Freed memory stays in the pool for later calls.
 */
#ifndef CSLICE_H
#define CSLICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t csl_status;
#define CSL_OK 0
#define CSL_ERR_INVALID_ARG 1   /* bad pointer, size, index, NaN/Inf, radius out of range */
#define CSL_ERR_OOM 2           /* a device or host allocation failed */
#define CSL_ERR_CUDA 3          /* a CUDA runtime call or kernel failed */
#define CSL_ERR_TIMEOUT 4       /* a bounded device-side wait gave up */
#define CSL_ERR_CAPACITY 5      /* a count exceeded a fixed-size buffer or int range */
#define CSL_ERR_NOT_READY 6     /* no GPU, or the object is not in a usable state */

#define CSL_MODE_PHYSICAL 0
#define CSL_MODE_RAW 1

/* Lattice parameters (Sec. 3.2). */
typedef struct csl_params {
    double R;                 /* kernel support; <= 0 selects 1.5 x the largest radius */
    double C;                 /* iso-value, > 0 (default 1 when 0 is passed)           */
    int32_t mode;             /* CSL_MODE_PHYSICAL or CSL_MODE_RAW                     */
    int32_t input_on_device;  /* 1: nodes/edges/radius are device pointers, 0: host    */
} csl_params;

typedef struct csl_lattice csl_lattice;   /* opaque; device-resident lattice */

typedef struct csl_lattice_info {
    int64_t n_nodes, n_edges;
    double R, C;
    int32_t mode, pad_;
    float bbox_lo[3], bbox_hi[3];   /* node bounding box (mm) */
    float max_dz;                   /* largest |v_e^z - v_s^z| over edges */
    float max_radius;
} csl_lattice_info;

/*
 * csl_lattice_upload -- copy a lattice to the GPU and prepare it for slicing.
 *   nodes_xyz  float[n_nodes][3]  node positions in mm (host or device, see
 *                                 params->input_on_device)
 *   edges_ij   int32[n_edges][2]  node indices of each edge's endpoints
 *   radius     float[n_edges]     per-edge radius (PHYSICAL) or weight (RAW)
 *   params     may be NULL (R = 1.5 max radius, C = 1, PHYSICAL, host input)
 *   stream     cudaStream_t or NULL
 *   out        receives the handle; release it with csl_lattice_free
 * Preparation (Sec. 4): each edge is ordered so that v_s^z <= v_e^z (Eq. 8),
 * turned into a 32-byte record (v_s, unit direction, length, weight) and the
 * records are sorted by v_s^z with a stable device radix sort.
 * Errors: INVALID_ARG for n_edges > 2^31 - 1, an index outside [0, n_nodes),
 * a non-finite coordinate or radius, radius <= 0, or (PHYSICAL) radius >= R.
 * The inputs are not retained; the library keeps its own device copy.
 * Synchronises the stream (to report validation errors).
 */
csl_status csl_lattice_upload(const float* nodes_xyz, int64_t n_nodes, const int32_t* edges_ij,
                              const float* radius, int64_t n_edges, const csl_params* params,
                              void* stream, csl_lattice** out);

/*
 * csl_lattice_upload_streamed -- the same lattice, kept in host memory (the
 * GPU form of the paper's out-of-core sweep, Sec. 4: only the edges near the
 * planes being sliced need to be in memory). The inputs are HOST arrays
 * (params->input_on_device must be 0). The nodes are copied to the device;
 * the edges are prepared in batches of at most batch_edges (0: 2^24) on the
 * device, each batch sorted by v_s^z there, and the sorted batches are merged
 * on the host into the order of one stable sort; the records stay in
 * page-locked host memory. csl_slice_layers then copies each chunk's z window
 * of the records to the device, so device memory holds the nodes and two
 * windows instead of the whole lattice; its results equal those of
 * csl_lattice_upload bit for bit. Such a lattice serves csl_slice_layers and
 * csl_lattice_get_info only; the other calls return NOT_READY. Errors as
 * csl_lattice_upload, plus INVALID_ARG for device inputs or batch_edges < 0.
 */
csl_status csl_lattice_upload_streamed(const float* nodes_xyz, int64_t n_nodes,
                                       const int32_t* edges_ij, const float* radius,
                                       int64_t n_edges, const csl_params* params,
                                       int64_t batch_edges, void* stream, csl_lattice** out);

/*
 * csl_lattice_update -- replace node positions and/or radii of an uploaded
 * lattice (same edges), e.g. inside a radius-tuning loop (Sec. 5.4).
 * nodes_xyz (float[n_nodes][3]) and radius (float[n_edges]) are device
 * pointers; either may be NULL to keep the current values. R is kept as it
 * was at upload. Re-sorts the records. Synchronises the stream.
 */
csl_status csl_lattice_update(csl_lattice* lat, const float* nodes_xyz, const float* radius,
                              void* stream);

csl_status csl_lattice_get_info(const csl_lattice* lat, csl_lattice_info* out);
void csl_lattice_free(csl_lattice* lat);

/* Slicing request (Sec. 4). */
#define CSL_SLICE_CONTOURS_ON_DEVICE 1   /* leave the contour arrays in device memory */
#define CSL_SLICE_EDGE_IDS 2             /* also return the grid-edge id of every vertex */
#define CSL_SLICE_NO_CONTOURS 4          /* field (and sigma_out) only; no marching squares */
#define CSL_SLICE_TIME_KERNELS 8         /* time each stage with CUDA events (csl_stats); the chunks
                                            then run one after another on the caller's stream */
#define CSL_SLICE_COUNT_PAIRS 16         /* count (pixel, layer, edge) pairs with a nonzero term */
#define CSL_SLICE_FUSED 32               /* footprint kernel with contours: the fused field and
                                            contour pass. The field kernel evaluates each tile with
                                            its next column and row and leaves the tile's crossing
                                            vertices (from Sigma in shared memory) and saddle bits
                                            instead of a Sigma plane: less device memory, the same
                                            contours bit for bit; without it (the default) a Sigma
                                            plane is written and marching squares reads it, which
                                            is faster when the field kernel is issue-bound */

/* Field kernels (Eq. 6-7 on the pixel grid; the results agree within FP32
 * rounding, and bit for bit at the same tile size):
 *   CSL_FIELD_BLOCK      every warp owns an 8 x 4-pixel block of a 16 x 16 tile
 *                        and sums, for each edge whose support can reach the
 *                        block, the term of all 32 pixels (suits supports of
 *                        many pixels);
 *   CSL_FIELD_FOOTPRINT  one warp per layer walks each edge's footprint in the
 *                        layer plane (the rows or columns of pixels within R of
 *                        its line), 32 footprint pixels per step (suits
 *                        supports of a few pixels).
 * CSL_FIELD_AUTO takes the footprint kernel on 32-pixel tiles when R is below
 * 10 pixels, else the block kernel. */
#define CSL_FIELD_AUTO 0
#define CSL_FIELD_BLOCK 1
#define CSL_FIELD_FOOTPRINT 2

typedef struct csl_slice_desc {
    double z0, dz;            /* layer k is the plane z = z0 + k dz                     */
    int32_t n_layers;         /* >= 0                                                   */
    int32_t nx, ny;           /* pixels per layer, 1 .. 32000 each                      */
    int32_t flags;            /* CSL_SLICE_* bits                                       */
    double x0, y0;            /* pixel (i, j) has its centre at (x0 + (i + 1/2) pixel,  */
    double pixel;             /*                                 y0 + (j + 1/2) pixel)  */
    float* sigma_out;         /* optional device float[n_layers][ny][nx]: Sigma per pixel */
    int32_t tile;             /* pixels per tile side: 0 (auto), 16 or 32 (32: footprint
                                 kernel only)                                            */
    int32_t slab;             /* layers per slab: 0 (auto), 1, 2, 4 or 8               */
    int32_t chunk_layers;     /* layers per streamed chunk: 0 (auto) or a multiple of slab */
    int16_t field_kernel;     /* CSL_FIELD_AUTO (0), CSL_FIELD_BLOCK or CSL_FIELD_FOOTPRINT */
    int16_t stage_records;    /* footprint kernel: records per staged copy, 0 (256) or a
                                 multiple of 32 up to 1024                               */
    uint32_t* mask_out;       /* optional device uint32[n_layers][ny][ceil(nx/32)]: the binary
                                 image of each layer (Sec. 4, the DLP mask): bit i % 32 of word
                                 [k][j][i / 32] is set when pixel (i, j) of layer k is inside
                                 (Sigma >= C); bits past nx are 0 */
    int64_t workspace_budget; /* 0: no limit. Else the bytes of device memory the call may hold
                                 besides the lattice (the paper slices in bounded memory, Sec. 4,
                                 6): one chunk in flight, a first chunk of two slabs measures the
                                 workspace per layer, the next chunks are sized to fit, and each
                                 chunk's contours go to the host as soon as they are done. Host
                                 contours only (not with CSL_SLICE_CONTOURS_ON_DEVICE), a
                                 device-resident lattice, no chunk_layers; the same results as
                                 without a budget. CAPACITY when one slab does not fit */
} csl_slice_desc;

/*
 * Contours of all layers. Loops are closed polygons with the inside of the
 * solid on their left (outer boundaries counter-clockwise with x right, y up).
 * The pixel grid is padded by one ring of outside samples, so every loop
 * closes. Within a layer, loops are listed by their smallest grid-edge id and
 * each loop starts at that edge; the grid edge from padded sample (I, J) to
 * (I+1, J) has id 2 (J (nx+2) + I) and the one to (I, J+1) has id
 * 2 (J (nx+2) + I) + 1, where padded sample (I, J) is pixel (I-1, J-1).
 * Each vertex is the zero of the linear interpolant of Sigma - C along its
 * grid edge; a saddle cell joins its inside corners when the mean of its four
 * corner values is >= C.
 */
/* Host arrays (on_device = 0) share one page-locked block, taken from a
 * per-process cache so that device-to-host copies run at the link's speed;
 * csl_contours_free returns the block to the cache (free blocks above 64 GiB
 * in total are released). Device arrays from csl_slice_layers are written in
 * place chunk by chunk: loop_vert_off, xy and edge_id grow behind reserved
 * address ranges (the driver's virtual memory management), so no copy of the
 * whole result is made; csl_contours_free releases them. */
typedef struct csl_contours {
    int32_t n_layers;
    int32_t on_device;        /* 1: the arrays below are device pointers           */
    int64_t n_loops;
    int64_t n_verts;
    int64_t* layer_loop_off;  /* [n_layers + 1] first loop of each layer            */
    int64_t* loop_vert_off;   /* [n_loops + 1] first vertex of each loop            */
    float* xy;                /* [n_verts][2] vertex positions in mm                */
    int32_t* edge_id;         /* [n_verts] grid-edge ids, or NULL without CSL_SLICE_EDGE_IDS */
} csl_contours;

/*
 * csl_slice_layers -- evaluate the field on every pixel of every layer,
 * threshold it at C and trace the contours.
 *   lat   lattice from csl_lattice_upload
 *   desc  slicing request; desc->sigma_out, when set, receives Sigma, and
 *         desc->mask_out, when set, the bit-packed inside mask
 *   out   receives the contours (library-owned; csl_contours_free); may be
 *         NULL with CSL_SLICE_NO_CONTOURS
 * Errors: INVALID_ARG for n_layers < 0, a non-finite dz, dz <= 0 (when n_layers > 1),
 * pixel <= 0, nx or ny outside [1, 32000], a non-finite origin, an
 * unsupported tile/slab/chunk value. CAPACITY when an internal count exceeds
 * 32-bit range per streamed chunk. Synchronises the stream.
 */
csl_status csl_slice_layers(csl_lattice* lat, const csl_slice_desc* desc, void* stream,
                            csl_contours** out);
void csl_contours_free(csl_contours* c);

/*
 * csl_contours_copy -- copy the arrays of c into caller buffers (each may be
 * NULL to skip it). dst_on_device: 1 if the destinations are device memory.
 * Sizes: layer_loop_off [n_layers + 1], loop_vert_off [n_loops + 1],
 * xy [2 n_verts], edge_id [n_verts] (only when c has edge ids).
 * Synchronises the stream.
 */
csl_status csl_contours_copy(const csl_contours* c, int64_t* layer_loop_off, int64_t* loop_vert_off,
                             float* xy, int32_t* edge_id, int32_t dst_on_device, void* stream);

/*
 * csl_contours_create -- device contours from HOST arrays in the layout of
 * csl_contours (for post-processing contours made elsewhere: simplification,
 * smoothing, zigzag infill). layer_loop_off [n_layers + 1] from 0 to n_loops
 * and loop_vert_off [n_loops + 1] from 0 to n_verts, both non-decreasing;
 * xy [2 n_verts] in mm (finite); edge_id [n_verts] grid-edge ids (>= 0) or
 * NULL. The library copies the arrays and owns the result (free with
 * csl_contours_free). Errors: INVALID_ARG (counts, offsets, non-finite
 * vertices, negative ids), OOM. Synchronises the stream.
 */
csl_status csl_contours_create(int32_t n_layers, int64_t n_loops, int64_t n_verts,
                               const int64_t* layer_loop_off, const int64_t* loop_vert_off,
                               const float* xy, const int32_t* edge_id, void* stream,
                               csl_contours** out);

/*
 * Zigzag infill of the contours (Sec. 6: the interior of each layer is filled
 * by a zigzag toolpath after its boundary contours). Scan lines
 * y_m = y0 + m spacing, m in [0, n_lines), the same in every layer (y_m is
 * computed in double and rounded once to float). A contour edge a -> b crosses
 * line m when min(a_y, b_y) <= y_m < max(a_y, b_y), decided in float, at
 * x = a_x + t (b_x - a_x), t = (y_m - a_y) / (b_y - a_y) in float. Along a line
 * the crossings sorted by x pair up into the inside segments. Each layer's
 * toolpath visits the lines in increasing m; on even lines its segments run
 * from low to high x in increasing x, on odd lines from high to low x in
 * decreasing x (the zigzag).
 *   contours  device contours (csl_slice_layers with CSL_SLICE_CONTOURS_ON_DEVICE)
 *   out       layer_seg_off [n_layers + 1] and seg [n_segments][3] = (x_from,
 *             x_to, y) in toolpath order, in mm (library-owned; csl_hatches_free);
 *             host page-locked blocks, or device memory with dst_on_device
 * Errors: INVALID_ARG (host contours, spacing <= 0, non-finite y0, n_lines < 0),
 * CAPACITY (n_layers * n_lines >= 2^32), CUDA (a line with an odd number of
 * crossings: contours that are not closed). Synchronises the stream.
 */
typedef struct csl_hatches {
    int32_t n_layers;
    int32_t on_device;
    int64_t n_segments;
    int64_t* layer_seg_off;   /* [n_layers + 1] first segment of each layer */
    float* seg;               /* [n_segments][3] x_from, x_to, y           */
} csl_hatches;
csl_status csl_hatch_layers(const csl_contours* contours, double y0, double spacing,
                            int32_t n_lines, int32_t dst_on_device, void* stream,
                            csl_hatches** out);
void csl_hatches_free(csl_hatches* h);

/*
 * Bins of one slab, for inspection: the edges (as sorted-record positions
 * mapped back to original edge ids, ascending) that the binner assigns to each
 * tile of the slab made of layers [first_layer, first_layer + n_slab_layers).
 * tile_off: host int64[ntx * nty + 1]; ids: host int32[capacity]. Returns the
 * number of ids in *n_ids (CAPACITY if it exceeds capacity). Tiles are
 * row-major, tile (tx, ty) covering pixels [tx T, tx T + T) x [ty T, ty T + T).
 */
csl_status csl_debug_slab_bins(csl_lattice* lat, const csl_slice_desc* desc, int32_t first_layer,
                               int32_t n_slab_layers, int64_t* tile_off, int32_t* ids,
                               int64_t capacity, int64_t* n_ids, void* stream);

/*
 * Density cells (Eq. 9): cell (ix, iy, iz), 0 <= i* < dims[*], is the cube
 * origin + h [i, i+1)^3; it is sampled at the m^3 points
 * origin + h (i + (k + 1/2) / m), k in [0, m) per axis.
 */
typedef struct csl_cells {
    double origin[3];
    double h;                 /* cell edge (mm), > 0                                    */
    int32_t dims[3];          /* cells per axis; dims[0] m, dims[1] m <= 32000          */
    int32_t m;                /* samples per cell axis: 1, 2, 4 or 8                    */
    double temperature;       /* T > 0 of the sigmoid (absolute; e.g. 0.01 C)           */
} csl_cells;

/*
 * csl_volume_fraction -- smoothed volume fraction of the solid in every cell:
 *   vf[iz][iy][ix] = (1/m^3) sum over the cell's samples p of
 *                    1 / (1 + exp(-(Sigma(p) - C) / T)),
 * the density of Eq. 9 with the Monte-Carlo hit count replaced by stratified
 * samples and a sigmoid, so that it is differentiable (radius tuning, Sec.
 * 5.4). vf_out: device float[dims[2]][dims[1]][dims[0]] (caller-owned).
 * Errors: INVALID_ARG for bad cells (see csl_cells) or NULL pointers.
 * Synchronises the stream.
 */
csl_status csl_volume_fraction(csl_lattice* lat, const csl_cells* cells, float* vf_out,
                               void* stream);

/*
 * csl_volume_fraction_backward -- gradient of a scalar loss L with respect to
 * every radius and node position, given grad_vf = dL/dvf (device, the layout
 * of vf_out). Sigma is recomputed (nothing is kept from the forward call).
 *   dL/drho_j = sum_c grad_vf_c (1/m^3) sum_p s(1-s)/T * I_j(p) * dw_j/drho_j
 *   dL/dv_i   = sum over the edges at node i of the same factor times
 *               w_j dI_j/d(endpoint)
 * with s the sigmoid at p, I_j the segment integral of Eq. 7 and w_j the
 * weight (PHYSICAL: dw/drho = w 5 rho / (R^2 - rho^2); RAW: 1). R and C are
 * held fixed.
 *   grad_radius  device float[n_edges]   (overwritten)
 *   grad_nodes   device float[n_nodes][3] (overwritten)
 * The sums run in a fixed order: results are deterministic.
 * Synchronises the stream.
 */
csl_status csl_volume_fraction_backward(csl_lattice* lat, const csl_cells* cells,
                                        const float* grad_vf, float* grad_radius,
                                        float* grad_nodes, void* stream);

/*
 * Batched slicing: many (lattice, slicing request) jobs -- lattices of uneven
 * size, or slab ranges of one lattice -- run as one CUDA graph whose field
 * stage is a single persistent launch. The paper slices one part at a time
 * (Sec. 4); batching is this library's own addition, so that many small
 * parts fill the GPU.
 *
 * csl_batch_create plans the batch: it runs every job once in the ordinary
 * way (reading the sizes the pipeline discovers: binner entries, crossings,
 * splitters, loops), keeps every buffer at those sizes, and captures a replay
 * of all jobs that reads nothing back into a CUDA graph: the binner and the
 * contour stages of the jobs run on parallel branches, and the field of all
 * jobs is one persistent kernel whose CTAs take (job, slab, tile) items from
 * a queue sorted longest tile list first (the block or the footprint kernel,
 * one for all jobs). With autotune set, it times the graph over a staged
 * search and keeps the fastest: first the field kernel and tile T (block on
 * 16-pixel tiles, footprint on 16- and 32-pixel tiles) at the default slab
 * depth; then, for the best of those, slab depth S in {2, 4, 8} x resident
 * CTAs per SM (2, 4, 6 for the block kernel; 2, 4 for the footprint kernel,
 * whose shared-memory planes bound residency); then, for the footprint
 * kernel, the records per staged copy K in {128, 256, 512}. The choice is
 * cached per process for the same job sizes; csl_batch_info lists every
 * timed candidate.
 *
 * csl_batch_run launches the graph on `stream` and waits for it. The jobs'
 * lattices are read at run time, so radii and node positions may change
 * between runs (csl_lattice_update), but every count must stay what the plan
 * saw: when the device finds another count it writes nothing out of range,
 * and the run returns CSL_ERR_CAPACITY (create the batch again). The results
 * of the last run stay in the batch: csl_batch_contours copies one job's
 * contours out, csl_batch_sigma gives the device address of its field.
 *
 * Lattices must outlive the batch, and must not be freed or re-uploaded
 * while it exists. Results are bit-identical to csl_slice_layers of each job
 * with the same slab depth (the same kernels sum the same terms in the same
 * order; the first plane of a slab is the origin of its FP32 z coordinates).
 */
typedef struct csl_batch csl_batch;   /* opaque */

typedef struct csl_batch_opts {
    int32_t autotune;         /* nonzero: time the candidates (field kernel and tile, slab,
                                 CTAs per SM, staging chunk) and keep the fastest          */
    int32_t slab;             /* without autotune: 0 (8, or less for short jobs) or 2, 4, 8 */
    int32_t ctas_per_sm;      /* without autotune: 0 (4) or 1 .. 6                     */
    int32_t branches;         /* parallel graph branches for binner and contours: 0 (8) or 1 .. 32 */
    int32_t field_kernel;     /* without autotune: CSL_FIELD_AUTO (the block kernel),
                                 CSL_FIELD_BLOCK or CSL_FIELD_FOOTPRINT                 */
    int32_t tile;             /* without autotune: 0 (16; 32 with the footprint kernel), 16, 32 */
    int32_t stage_records;    /* without autotune: 0 (256) or a multiple of 32 up to 1024
                                 (footprint kernel)                                      */
    int32_t reserved_;
} csl_batch_opts;

#define CSL_BATCH_MAX_CANDIDATES 16
typedef struct csl_batch_info {
    int32_t n_jobs;
    int32_t slab;             /* chosen slab depth                                       */
    int32_t ctas_per_sm;      /* chosen persistent CTAs per SM                           */
    int32_t from_cache;       /* 1: the choice came from the per-process cache           */
    int64_t n_items;          /* (job, slab, tile) items of the field queue              */
    int64_t n_pairs;          /* binner entries over all jobs                            */
    int64_t n_crossings;      /* contour vertices over all jobs                          */
    int64_t n_loops;
    int64_t graph_nodes;
    int64_t pixel_evals;      /* sum over jobs of n_layers * nx * ny                     */
    double plan_ms;           /* host time of the planning runs                          */
    double tune_ms;           /* host time of the autotuning                             */
    int32_t n_candidates;     /* autotuned candidates and their best graph time          */
    int32_t cand_slab[CSL_BATCH_MAX_CANDIDATES];
    int32_t cand_ctas[CSL_BATCH_MAX_CANDIDATES];
    float cand_ms[CSL_BATCH_MAX_CANDIDATES];
    int32_t cand_kernel[CSL_BATCH_MAX_CANDIDATES];   /* CSL_FIELD_BLOCK / _FOOTPRINT */
    int32_t cand_tile[CSL_BATCH_MAX_CANDIDATES];
    int32_t cand_stage[CSL_BATCH_MAX_CANDIDATES];
    int32_t field_kernel;     /* chosen field kernel, tile and staging chunk              */
    int32_t tile;
    int32_t stage_records;
    int32_t reserved_;
} csl_batch_info;

/*
 * csl_batch_create -- plan (and, with opts->autotune, tune) a batch.
 *   lats[j], descs[j]  job j: a lattice and a slicing request as for
 *                      csl_slice_layers; only z0, dz, n_layers (>= 1), nx, ny,
 *                      x0, y0, pixel and the CSL_SLICE_EDGE_IDS flag are used.
 *                      A job must fit one streamed chunk (all of its layers'
 *                      Sigma at once, fewer than 2^27 contour edge words).
 *   n_jobs             >= 1
 *   opts               may be NULL (no autotuning, defaults)
 * Errors: INVALID_ARG (a NULL lattice, a bad request, a job too large for one
 * chunk), OOM, CUDA. Synchronises the stream.
 */
csl_status csl_batch_create(csl_lattice* const* lats, const csl_slice_desc* descs, int32_t n_jobs,
                            const csl_batch_opts* opts, void* stream, csl_batch** out);
/* Launch the graph on stream and wait; CSL_ERR_CAPACITY if a count changed. */
csl_status csl_batch_run(csl_batch* b, void* stream);
/* Contours of job j from the last run (csl_contours_free; dst_on_device as
 * CSL_SLICE_CONTOURS_ON_DEVICE). */
csl_status csl_batch_contours(const csl_batch* b, int32_t job, int32_t dst_on_device,
                              csl_contours** out);
/* Device address of job j's Sigma, float[n_layers][ny][nx], owned by the batch
 * and overwritten by every run. */
csl_status csl_batch_sigma(const csl_batch* b, int32_t job, float** out);
csl_status csl_batch_get_info(const csl_batch* b, csl_batch_info* out);
void csl_batch_free(csl_batch* b);

/*
 * csl_field_layers_static -- Sigma on the layers of desc for a lattice given
 * as raw device arrays, WITHOUT allocating any memory. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory, e.g. an application that plans all of its device memory up front (a
 * fixed budget or its own allocator that forbids outside allocations), or one
 * that must not take the implicit device synchronisation of cudaMalloc and
 * cudaFree. It calls no cudaMalloc, cudaFree or allocating library routine.
 *   nodes_xyz, edges_ij, radius  device arrays as in csl_lattice_upload
 *   R                            support radius, > 0 (no default here)
 *   C, mode                      as csl_params (C = 0 means 1)
 *   desc                         z0, dz, n_layers (<= 65535), x0, y0, nx, ny,
 *                                pixel are used; everything else is ignored
 *   sigma_out                    device float[n_layers][ny][nx] (caller-owned)
 * Its only scratch is a fixed static device array: 256 bytes plus 32 bytes per
 * edge for at most CSL_STATIC_MAX_EDGES edges (8 MiB + 256 bytes); larger
 * inputs are rejected with CSL_ERR_CAPACITY. The array is reserved when the
 * library's module is loaded on a device, which with CUDA's lazy loading (the
 * default) happens at the first call on that device, and it stays reserved
 * until the process exits. That first call also looks up the array's device
 * address (cudaGetSymbolAddress), and the module load may allocate and
 * synchronise: callers with a fixed memory plan make the first call during
 * set-up, and always before any stream capture. The address is cached per
 * CUDA context, so a call after cudaDeviceReset looks it up again. Every call
 * reuses the array (its status word is cleared, its records rewritten): calls
 * whose GPU work overlaps, on other streams or host threads, race on it and
 * must be serialised by the caller.
 * Edges are summed in edge order (not z order), so values agree with
 * csl_slice_layers within FP32 rounding, not bit for bit.
 * Errors: INVALID_ARG for the csl_lattice_upload and csl_slice_layers input
 * errors (bad index, a non-finite node coordinate (of any node) or radius,
 * radius <= 0 or >= R in PHYSICAL mode; a non-finite dz, even for one layer),
 * the device-side ones reported after the GPU work, in which case sigma_out is
 * unspecified.
 * Synchronises the stream.
 */
#define CSL_STATIC_MAX_EDGES 262144
csl_status csl_field_layers_static(const float* nodes_xyz, int64_t n_nodes, const int32_t* edges_ij,
                                   const float* radius, int64_t n_edges, double R, double C,
                                   int32_t mode, const csl_slice_desc* desc, float* sigma_out,
                                   void* stream);

/* Statistics of the last csl_slice_layers call on this thread. */
typedef struct csl_stats {
    int64_t candidate_pairs;  /* (slab, tile, edge) entries produced by the binner */
    int64_t crossings;        /* marching-squares vertices                          */
    int64_t loops;
    int64_t chunks;
    int64_t device_bytes_peak;/* largest workspace held at once                     */
    int64_t kernel_launches;  /* kernels this library launched during the call      */
    int64_t field_launches;   /* launches of the field kernel                       */
    double field_ms;          /* their summed CUDA-event time (CSL_SLICE_TIME_KERNELS) */
    int64_t contributing_pairs; /* pairs with a nonzero term (CSL_SLICE_COUNT_PAIRS) */
    double bin_ms;            /* CUDA-event time of the binner (CSL_SLICE_TIME_KERNELS) */
    double contour_ms;        /* ... of marching squares and loop assembly            */
    double output_ms;         /* ... of gathering the chunks into the result          */
    int64_t evaluated_terms;  /* terms the field kernel evaluated (CSL_SLICE_COUNT_PAIRS) */
    int64_t window_records;   /* records the binner examined (the slabs' z windows, summed) */
    /* the plan the call resolved: field kernel (CSL_FIELD_BLOCK or CSL_FIELD_FOOTPRINT),
       tile side, slab depth, records per staged copy, fused pass (0 or 1) */
    int32_t field_kernel, tile, slab, stage_records;
    int32_t fused, reserved_;
} csl_stats;
csl_status csl_last_stats(csl_stats* out);

/*
 * csl_support_metrics -- self-support metrics of the lattice (Sec. 5.3):
 * theta_j = arccos |u_j . t_P| per edge (Eq. 11); an edge with theta_j <= alpha
 * is fully self-supported; g(theta) = sum_{i<6} a_i theta^i for theta > alpha,
 * else 0 (Eq. 12); *gamma = sum over unsupported edges of r_j L_j g(theta_j) /
 * sum over all edges of r_j L_j (Eq. 13); *psi = 100 x sum over supported edges
 * of L_j / sum of L_j (Eq. 14). r_j is the edge's radius value as uploaded.
 *   t_p     host double[3], the printing direction (any nonzero length)
 *   alpha   the self-supporting angle in [0, pi/2] (the paper uses pi/4)
 *   coeffs  host double[6] a_0..a_5, or NULL for the paper's quintic for pi/4
 * Sums in double in a fixed order (deterministic). Synchronises the stream.
 */
csl_status csl_support_metrics(const csl_lattice* lat, const double* t_p, double alpha,
                               const double* coeffs, double* gamma, double* psi, void* stream);

/*
 * csl_debug_wait_timeout -- test of the bounded device waits: launches one
 * block that waits, with the field kernel's mbarrier wait, on a barrier that
 * nothing arms, giving up after `polls` polls (1 .. 2^22). Returns
 * CSL_ERR_TIMEOUT when the wait gave up and reported it (the expected result);
 * the device stays usable. The paper has no counterpart.
 */
csl_status csl_debug_wait_timeout(uint32_t polls, void* stream);

/*
 * csl_measure_fp32_peak -- FP32 throughput of the device, measured with a
 * kernel of independent FFMA chains at full occupancy (best of 5 timed
 * launches after one warm-up). A measurement helper for the roofline of the
 * ALU-bound kernels; not part of the method. *tflops receives TFLOP/s (FFMA =
 * 2 flops); *sm_clock_ghz (may be NULL) the device's nominal maximum SM clock.
 * Synchronises the stream.
 */
csl_status csl_measure_fp32_peak(double* tflops, double* sm_clock_ghz, void* stream);

/*
 * csl_simplify_contours -- topology-preserving simplification of device
 * contours (the paper simplifies its marching-squares boundaries without
 * creating intersections, Sec. 4). A vertex on grid edge e, at an odd
 * position of a loop of >= 5 vertices, is dropped when neither grid cell
 * beside e has a crossing on an edge other than the loop's own (so both cells
 * hold only this loop, and the chord joining its neighbours stays in their
 * convex 1 x 2 block) and it lies within tol (mm) of that chord (FP64). Loops,
 * their order and their heads are kept; every loop keeps >= 3 vertices; no two
 * segments of a layer cross if none did. in: device contours with edge ids
 * (CSL_SLICE_CONTOURS_ON_DEVICE | CSL_SLICE_EDGE_IDS) of an nx x ny grid;
 * out: new device contours with edge ids (csl_contours_free). Errors:
 * INVALID_ARG (host contours, no edge ids, nx/ny out of range, tol < 0),
 * CAPACITY (the per-layer edge bitmaps above 16 GiB), OOM. Synchronises.
 */
csl_status csl_simplify_contours(const csl_contours* in, int32_t nx, int32_t ny, double tol,
                                 void* stream, csl_contours** out);

/*
 * csl_smooth_contours -- topology-preserving smoothing of device contours, in
 * place (the paper smooths its marching-squares boundaries without creating
 * intersections, Sec. 4). Every vertex slides along its own grid edge of the
 * padded nx x ny sample grid (pixel size `pixel`, first pixel centre at
 * (x0 + pixel/2, y0 + pixel/2)): in each of `iterations` Jacobi steps its
 * free coordinate a (x on a horizontal edge, y on a vertical one) becomes
 * a + lambda (m - a), m the mean of that coordinate at its loop neighbours,
 * clamped to the edge's [margin, 1 - margin] part, in float32 with every
 * operation rounded on its own (m = 0.5 (a_p + a_s); a + lambda (m - a); the
 * edge's first sample lo = (x0 - pixel/2) + I pixel; lo + margin pixel and
 * lo + (1 - margin) pixel, lambda and the two margins rounded once from
 * double); the other coordinate, the edge ids and all offsets are unchanged;
 * loops of fewer than 3 vertices stay as they are. Every segment stays
 * inside its grid cell (or the 1 x 2 block of a vertex that simplification
 * dropped), so no two segments can come to cross. c: device contours with
 * edge ids of that grid. Errors: INVALID_ARG (host contours, no edge ids, an
 * edge id outside the grid, nx/ny outside [1, 32000], pixel <= 0, lambda
 * outside [0, 1], margin outside (0, 1/2], iterations outside [0, 10000]) with
 * c unchanged; CAPACITY (more than 2^31 - 1 loops); OOM. Synchronises.
 */
csl_status csl_smooth_contours(csl_contours* c, double x0, double y0, double pixel, int32_t nx,
                               int32_t ny, double lambda, double margin, int32_t iterations,
                               void* stream);

/* ---- ray casting of the implicit solid (a depth image, no mesh) --------- */

typedef struct csl_camera {
    double eye[3], target[3], up[3];   /* pinhole camera; up fixes the roll */
    double fov_y;          /* vertical field of view, radians, in (0, pi) */
    int32_t width, height; /* pixels; pixel (i, j), j the row from the top */
    double step;           /* sample spacing along a ray (mm), > 0 */
    int32_t refine;        /* halvings of the step that holds the surface, 0..60 */
    int32_t reserved;
} csl_camera;

/*
 * csl_render_depth -- the distance along each pixel's unit ray to the solid
 * {Sigma >= C} (Sec. 3; the paper shows its lattices by ray tracing the
 * implicit function directly). A ray is sampled at t_in + k * step from where
 * it enters the lattice's box grown by R; the first sample with Sigma >= C is
 * refined by `refine` halvings of the preceding step; no such sample: +inf.
 * Features thinner than a step can be missed. The struts are binned into a
 * uniform grid of cells of edge >= 2R (empty cells are skipped). depth: DEVICE
 * float [height][width]. Errors: INVALID_ARG (camera, sizes, a step giving
 * more than 2^24 samples across the grown box), CAPACITY (more than 2^31
 * strut-cell pairs), OOM. Synchronises the stream.
 */
csl_status csl_render_depth(const csl_lattice* lat, const csl_camera* cam, float* depth,
                            void* stream);

/* ---- vertex position optimisation for self-support (Sec. 5.3.2) ---------- */

typedef struct csl_po_params {
    double t_p[3];        /* printing direction (nonzero; normalised here) */
    double alpha;         /* self-supporting angle in [0, pi/2] (pi/4 in the paper) */
    double a[6];          /* g(theta) = sum_i a_i theta^i for theta > alpha (Eq. 12) */
    double step;          /* first trial step, in units of tau0 (> 0) */
    double ball;          /* radius of the allowed ball around the initial position, in tau0 */
    double min_volume;    /* an incident tetrahedron keeps this share of its volume, [0, 1) */
    int32_t backtracks;   /* step halvings per visit, 0..60 */
    int32_t max_rounds;   /* 0..100000 */
} csl_po_params;

typedef struct csl_po_result {
    int32_t rounds;        /* rounds run (the last one moved nothing, unless max_rounds) */
    int32_t n_colours;     /* colours of the greedy colouring */
    int64_t moves;         /* accepted moves over all rounds */
    double gamma_before, psi_before, gamma_after, psi_after;   /* Eq. 13-14 of the mesh's edges */
    double host_ms;        /* time in the host-side setup (edges, adjacency, boundary, colouring) */
    double wall_ms;        /* time of the whole call */
} csl_po_result;

/*
 * csl_support_optimize -- vertex re-positioning for self-support (Sec. 5.3.2,
 * Eq. 16-17). Every interior vertex of the tetrahedral mesh moves along
 * -grad J(v), J(v) = sum_{e at v} r_e L_e g(theta_e) / sum_{e at v} r_e L_e,
 * theta_e = arccos |u_e . t_P| (Eq. 11), by step * tau0 halved up to
 * `backtracks` times until the new position lies within ball * tau0 of the
 * initial one (tau0: the initial distance to the faces opposite the vertex, the
 * inscribed sphere of Eq. 17), keeps every incident tetrahedron's orientation
 * and min_volume of its volume, and lowers J. Vertices on the mesh boundary
 * stay. The paper's one-by-one order is a greedy colouring (vertex order,
 * smallest free colour): colour by colour, vertices by index; each colour is
 * one parallel step with the result of the sequential sweep. Rounds repeat
 * until none moves or max_rounds. FP64 throughout.
 * nodes: HOST float [n_nodes][3], updated in place; tets: HOST int32
 * [n_tets][4]; radius: HOST float per edge of the distinct tetrahedron edges
 * sorted by (smaller, larger) node id, or NULL for equal radii;
 * moves_per_round: HOST int32 [max_rounds] or NULL. Errors: INVALID_ARG
 * (index out of range, non-finite value, parameter out of range), CAPACITY.
 * Synchronises the stream.
 */
csl_status csl_support_optimize(float* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                                const float* radius, const csl_po_params* p, void* stream,
                                csl_po_result* out, int32_t* moves_per_round);

/* ---- density matching of a tetrahedral lattice (Sec. 5.5) ---------------- */

/* Target densities on a voxel grid: voxel (i, j, k) is the box origin + h *
 * ([i, i+1] x [j, j+1] x [k, k+1]); target is a HOST array [nz][ny][nx]. */
typedef struct csl_voxels {
    double origin[3];
    double h;               /* > 0 */
    int32_t dims[3];        /* nx, ny, nz >= 1, product < 2^31 */
    const float* target;    /* finite */
} csl_voxels;

typedef struct csl_dm_params {
    float r_min;        /* smallest printable radius (> 0); the base radius is r0 = 2 r_min */
    float R;            /* support radius, > 4 r_min (the doubled base radius); 0: 6 r_min */
    float C;            /* iso-value, > 0 */
    float temperature;  /* T / C of the smoothed indicator, > 0 (0.01 in the volume fraction) */
    int32_t tet_n;      /* n: n^3 samples per tetrahedron, 1..16 */
    int32_t vox_m;      /* m: m^3 samples per voxel, 1..16 */
    int32_t max_depth;  /* subdivision levels, 0..8 */
    int32_t iters;      /* bisection halvings, 1..40 */
} csl_dm_params;

/* Result of csl_density_match, host memory owned by the library (free with
 * csl_dm_result_free). Nodes: the input nodes, then the midpoints in creation
 * order. Edges: the unsplit edges (both node ids, smaller first) in creation
 * order, with their radii r0 * ratio. Tetrahedra: the leaves in creation order
 * (children follow all tetrahedra of the previous level), with depth, target
 * (Step 1), rho_star (density with the doubled radius) and ratio (Step 3). */
typedef struct csl_dm_result {
    int64_t n_nodes;
    float* nodes;            /* [n_nodes][3] */
    int64_t n_edges;
    int32_t* edges;          /* [n_edges][2] */
    float* radius;           /* [n_edges] */
    float* step3_ratio;      /* [n_edges]: the ratio before the voxel check */
    int64_t n_tets;
    int32_t* tets;           /* [n_tets][4] */
    int32_t* tet_depth;      /* [n_tets] */
    double* tet_target;      /* [n_tets] */
    float* tet_rho_star;     /* [n_tets] */
    float* tet_ratio;        /* [n_tets] */
    int64_t n_voxels;
    float* voxel_ratio;      /* [nz][ny][nx]; NaN where no edge meets the voxel */
    int64_t n_subdivided;    /* tetrahedra split over all levels */
    double host_ms;          /* time in the host-side topology edits and bookkeeping */
    double wall_ms;          /* time of the whole call */
} csl_dm_result;

/*
 * csl_density_match -- builds a lattice matching target densities from a
 * tetrahedral mesh (Sec. 5.5, the subdivision and radius-tuning operators and
 * the four steps):
 *   1. target of a tetrahedron = the largest target of the voxels whose
 *      centres it contains (closed test, FP64 determinants); with none, the
 *      trilinear interpolation of the voxel-centre values at its centroid;
 *   2. rho* = its density with the doubled radius 2 r0 on its six edges; while
 *      rho* < target (and depth < max_depth) it is cut 1:8 at its edges'
 *      midpoints (float32), the inner octahedron along its shortest diagonal;
 *      a split edge is replaced by its halves everywhere;
 *   3. every leaf bisects the common ratio s in [1/2, 2] of its six edges'
 *      radii r0 s for its target; an edge takes the smallest ratio of the
 *      leaves containing it;
 *   4. every voxel bisects a common ratio for the edges meeting it (closed
 *      segment-box test, FP64), the other struts at their Step-3 radii; an
 *      edge keeps the smaller of its ratio and the voxel's.
 * A density is the mean of sigma((Sigma - C) / (temperature C)) at n^3
 * equal-volume samples of the tetrahedron (centroids of its Kuhn subdivision)
 * or m^3 stratified samples of the voxel (Eq. 9), Sigma with the PHYSICAL
 * weights of radius r (Sec. 3.2); a tetrahedron's density uses its own six
 * struts. nodes [n_nodes][3], tets [n_tets][4]: HOST arrays (copied). The
 * densities, bisections and the voxel pass run on the device; the topology
 * of the subdivision is edited on the host between levels. Errors:
 * INVALID_ARG (index out of range, non-finite value, parameter out of range),
 * CAPACITY (more than 2^27 tetrahedra or 2^31 voxel-edge pairs), OOM.
 * Synchronises the stream.
 */
csl_status csl_density_match(const float* nodes, int64_t n_nodes, const int32_t* tets,
                             int64_t n_tets, const csl_voxels* vox, const csl_dm_params* p,
                             void* stream, csl_dm_result** out);
void csl_dm_result_free(csl_dm_result* r);

const char* csl_last_error(void);
const char* csl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CSLICE_H */
