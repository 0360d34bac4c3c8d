// Device-resident lattice (internal layout).
#pragma once

#include "common.cuh"

// One edge after preparation, in the order of its lower endpoint's z.
// 32 bytes: two float4 loads.
struct __align__(16) csl_rec {
    float ax, ay, az;   // v_s, the endpoint with the smaller z (Eq. 8)
    float ux;           // unit direction v_s -> v_e
    float uy, uz;
    float len;          // |v_e - v_s|
    float w;            // weight r_j of Eq. 6
};

struct csl_lattice {
    int64_t n_nodes = 0, n_edges = 0;
    double R = 0, C = 1;
    int32_t mode = CSL_MODE_PHYSICAL;
    csl::DevBuf nodes;    // float [n_nodes][3]
    csl::DevBuf edges;    // int32 [n_edges][2]
    csl::DevBuf radius;   // float [n_edges]
    csl::DevBuf rec;      // csl_rec [n_edges], sorted by v_s^z
    csl::DevBuf bxy;      // float4 [n_edges] (v_s^x, v_s^y, v_e^x, v_e^y), exact inputs
    csl::DevBuf zlo;      // float [n_edges] v_s^z, ascending
    csl::DevBuf zhi;      // float [n_edges] v_e^z
    csl::DevBuf sid;      // uint32 [n_edges]: original edge id | (endpoints swapped) << 31
    csl::DevBuf node_csr_off;  // int32 [n_nodes + 1] (built on first backward)
    csl::DevBuf node_csr;      // uint32 [2 n_edges]: sorted position << 1 | end (0 = v_s)
    csl::DevBuf status;        // uint32: ST_TIMEOUT when a device wait gave up
    float bbox_lo[3] = {0, 0, 0}, bbox_hi[3] = {0, 0, 0};
    float max_dz = 0, max_radius = 0;
};

namespace csl {
// (Re)builds rec/zlo/zhi/sid from nodes/edges/radius; validates the input.
void prepare_lattice(csl_lattice* L, bool recompute_R, cudaStream_t s);
}  // namespace csl
