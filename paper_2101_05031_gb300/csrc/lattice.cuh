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
    // A host-resident lattice (csl_lattice_upload_streamed) keeps the prepared
    // arrays below in page-locked host memory, in the order rec/zlo give; only
    // nodes and status live on the device, and slicing copies each chunk's
    // z window of them to the device.
    bool host_resident = false;
    csl_rec* h_rec = nullptr;
    float4* h_bxy = nullptr;
    float* h_zlo = nullptr;
    float* h_zhi = nullptr;
    uint32_t* h_sid = nullptr;
    ~csl_lattice() {
        void* blocks[] = {h_rec, h_bxy, h_zlo, h_zhi, h_sid};
        for (void* b : blocks)
            if (b) csl::host_block_free(b);
    }
};

namespace csl {
// (Re)builds rec/zlo/zhi/sid from nodes/edges/radius; validates the input.
void prepare_lattice(csl_lattice* L, bool recompute_R, cudaStream_t s);
// The same preparation for a host-resident lattice: L->nodes on the device,
// the edges and radii in host memory, at most `batch` edges on the device at
// a time; every batch is sorted on the device and the sorted batches are
// merged on the host in the order of the single sort.
void prepare_lattice_streamed(csl_lattice* L, const int32_t* edges, const float* radius,
                              int64_t batch, cudaStream_t s);
}  // namespace csl
