// The tetrahedral lattice of density matching (Sec. 5.5) on the device: its
// nodes, edges (with midpoints and halves once split) and tetrahedra, and the
// level-wise 1:8 subdivision (density_mesh.cu).
//
// Numbering follows the sequential definition, in which the tetrahedra of a
// level are visited in order and each split appends at once:
//  - the input's edges are numbered in (smaller, larger) node-id order;
//  - a split of tetrahedron t first splits its six edges in local order (an
//    edge split for the first time appends its midpoint node and then its two
//    halves (a, m), (m, b)), then appends its eight children, each with its
//    six edges in local order (an edge met for the first time is appended).
// On the device every split tetrahedron r of a level (in visiting order) owns
// 6 midpoint slots (6 r + k) and 60 edge slots (60 r + j: j = 2k, 2k + 1 the
// halves of local edge k, j = 12 + 6c + e edge e of child c); an item is
// created by the smallest slot that meets it, and prefix sums over the
// creators' flags give the ids the sequential visit gives.
#pragma once

#include "common.cuh"

namespace csl {

struct DevMesh {
    int64_t n_nodes = 0, n_edges = 0, n_tets = 0;
    DevBuf xyz;     // float [3 per node]
    DevBuf ekey;    // uint64 per edge: smaller node << 32 | larger node
    DevBuf mid;     // int32 per edge: midpoint node once split, else -1
    DevBuf half;    // int2 per edge: its halves once split, else (-1, -1)
    DevBuf tv;      // int4 per tetrahedron: its nodes
    DevBuf te;      // int32 [6 per tetrahedron]: its edges in local order
    DevBuf depth;   // int32 per tetrahedron
    DevBuf leaf;    // uint8 per tetrahedron
    DevBuf hkey, hval;   // edge key -> id (open addressing, linear probing)
    int64_t hcap = 0;
    DevBuf status;  // uint32: ST_CAPACITY when a table ran full
};

// The input mesh (host arrays, validated by the caller).
void mesh_init(DevMesh& m, const float* nodes, int64_t n_nodes, const int32_t* tets,
               int64_t n_tets, cudaStream_t s);

// float4 corners (xyz, 0) of tetrahedra [t0, t0 + n), 4 per tetrahedron.
void mesh_corners(const DevMesh& m, int64_t t0, int64_t n, float4* out, cudaStream_t s);

// Splits the flagged tetrahedra among [t0, t0 + n) (split: uint32 0 / 1 per
// tetrahedron of the range, device) into their 8 children each, appended in
// order at the end (ids n_tets .. n_tets + 8 n_split - 1). Returns n_split.
int64_t mesh_subdivide(DevMesh& m, int64_t t0, int64_t n, const uint32_t* split, cudaStream_t s);

// The final lattice: the unsplit edges (segments) in id order and the leaves
// in id order.
struct MeshFinal {
    int64_t n_seg = 0, n_leaf = 0;
    DevBuf segs;     // uint32 edge id per segment
    DevBuf seg_of;   // uint32 per edge: its segment index (unsplit edges only)
    DevBuf leaves;   // uint32 tetrahedron id per leaf
};
void mesh_finalize(const DevMesh& m, MeshFinal& f, cudaStream_t s);

// Step 3's rule: ratio_bits[seg] = min over the leaves whose edges contain the
// segment of their ratio (float bits of positive values; the caller starts
// them at +inf). tet_ratio: float per tetrahedron id.
void mesh_edge_min(const DevMesh& m, const MeshFinal& f, const float* tet_ratio,
                   uint32_t* ratio_bits, cudaStream_t s);

// Segment end points (float4 xyz, 0), in segment order.
void mesh_segment_points(const DevMesh& m, const MeshFinal& f, float4* sa, float4* sb,
                         cudaStream_t s);

// Gathers of the final arrays (device): edges of the segments (2 int32 each),
// and per leaf its nodes (4 int32), depth, and the tetrahedron-indexed values.
void mesh_gather_final(const DevMesh& m, const MeshFinal& f, int32_t* edges, int32_t* tets,
                       int32_t* depth, const double* t_target, double* target,
                       const float* t_rho, float* rho, const float* t_ratio, float* ratio,
                       cudaStream_t s);

}  // namespace csl
