// Level-wise 1:8 subdivision of a tetrahedral lattice on the device (Sec. 5.5,
// the subdivision operator), with the numbering of the sequential definition
// (density_mesh.cuh): per level, a prefix sum over the split flags orders the
// split tetrahedra; each claims its midpoint and edge slots; the smallest slot
// that meets an item creates it (atomicMin on the item), and prefix sums over
// the creators' flags number the new nodes and edges.
#include <algorithm>

#include "density_mesh.cuh"

namespace csl {
namespace {

constexpr uint64_t kEmptyKey = ~0ull;

// local edge e of a tetrahedron joins corners la(e) < lb(e):
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
__host__ __device__ __forceinline__ int la(int e) { return (0x211000 >> (4 * e)) & 0xf; }
__host__ __device__ __forceinline__ int lb(int e) { return (0x332321 >> (4 * e)) & 0xf; }

__device__ __forceinline__ int corner(const int4 v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

__device__ __forceinline__ uint64_t key_of(int a, int b) {
    const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    return ((uint64_t)lo << 32) | hi;
}

__device__ __forceinline__ uint64_t mix(uint64_t k) {   // a 64-bit finaliser
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return k;
}

// Slot of key k (or -1 when absent).
__device__ __forceinline__ int64_t table_find(const uint64_t* __restrict__ keys, uint64_t mask,
                                              uint64_t k) {
    uint64_t i = mix(k) & mask;
    for (uint64_t n = 0; n <= mask; ++n) {
        const uint64_t q = keys[i];
        if (q == k) return (int64_t)i;
        if (q == kEmptyKey) return -1;
        i = (i + 1) & mask;
    }
    return -1;
}

// Slot of key k, inserted when absent (-1 when the table is full).
__device__ __forceinline__ int64_t table_insert(uint64_t* keys, uint64_t mask, uint64_t k) {
    uint64_t i = mix(k) & mask;
    for (uint64_t n = 0; n <= mask; ++n) {
        const unsigned long long prev =
            atomicCAS(reinterpret_cast<unsigned long long*>(keys + i), kEmptyKey, k);
        if (prev == kEmptyKey || prev == k) return (int64_t)i;
        i = (i + 1) & mask;
    }
    return -1;
}

__global__ void k_hash_build(const uint64_t* __restrict__ ekey, int64_t n, uint64_t* hkey,
                             int32_t* hval, uint64_t mask, uint32_t* status) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = table_insert(hkey, mask, ekey[e]);
        if (i < 0) atomicOr(status, ST_CAPACITY);
        else hval[i] = (int32_t)e;
    }
}

// ---- input mesh ----

// event q = 6 t + e: the larger node of local edge e (first sort key)
__global__ void k_init_events(const int4* __restrict__ tv, int64_t n_tets,
                              uint32_t* __restrict__ key1, uint32_t* __restrict__ idx) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 6 * n_tets;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int4 v = tv[q / 6];
        const int e = (int)(q % 6);
        key1[q] = (uint32_t)max(corner(v, la(e)), corner(v, lb(e)));
        idx[q] = (uint32_t)q;
    }
}

// the smaller node of the event at sorted place p (second, stable sort key)
__global__ void k_init_key2(const int4* __restrict__ tv, const uint32_t* __restrict__ idx,
                            int64_t n, uint32_t* __restrict__ key2) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q = idx[p];
        const int4 v = tv[q / 6];
        const int e = (int)(q % 6);
        key2[p] = (uint32_t)min(corner(v, la(e)), corner(v, lb(e)));
    }
}

__device__ __forceinline__ uint64_t event_key(const int4* __restrict__ tv, uint32_t q) {
    const int4 v = tv[q / 6];
    const int e = (int)(q % 6);
    return key_of(corner(v, la(e)), corner(v, lb(e)));
}

__global__ void k_init_unique(const int4* __restrict__ tv, const uint32_t* __restrict__ idx,
                              int64_t n, uint32_t* __restrict__ flag) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = (p == 0 || event_key(tv, idx[p]) != event_key(tv, idx[p - 1])) ? 1u : 0u;
}

__global__ void k_init_edges(const int4* __restrict__ tv, const uint32_t* __restrict__ idx,
                             const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank,
                             int64_t n, uint64_t* __restrict__ ekey, int32_t* __restrict__ te) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = (int32_t)(rank[p] + flag[p]) - 1;   // the run's first place
        if (flag[p]) ekey[id] = event_key(tv, idx[p]);
        te[idx[p]] = id;
    }
}

__global__ void k_corners(const int4* __restrict__ tv, const float* __restrict__ xyz, int64_t t0,
                          int64_t n, float4* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 4 * n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int v = corner(tv[t0 + q / 4], (int)(q % 4));
        out[q] = make_float4(xyz[3 * (int64_t)v], xyz[3 * (int64_t)v + 1],
                             xyz[3 * (int64_t)v + 2], 0.0f);
    }
}

// ---- one level ----

// sidx[rank] = t0 + i for the split tetrahedra of the range
__global__ void k_list(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank,
                       int64_t n, int64_t base, uint32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[rank[i]] = (uint32_t)(base + i);
}

// midpoint slot q = 6 r + k: the first slot that meets a not yet split edge
__global__ void k_mid_claim(const uint32_t* __restrict__ sidx, int64_t n_split,
                            const int32_t* __restrict__ te, const int32_t* __restrict__ mid,
                            int32_t* __restrict__ first) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 6 * n_split;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = te[6 * (int64_t)sidx[q / 6] + q % 6];
        if (mid[x] < 0) atomicMin(first + x, (int32_t)q);
    }
}

__global__ void k_mid_flags(const uint32_t* __restrict__ sidx, int64_t n_split,
                            const int32_t* __restrict__ te, const int32_t* __restrict__ mid,
                            const int32_t* __restrict__ first, uint32_t* __restrict__ flag) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 6 * n_split;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = te[6 * (int64_t)sidx[q / 6] + q % 6];
        flag[q] = (mid[x] < 0 && first[x] == (int32_t)q) ? 1u : 0u;
    }
}

// the creators' midpoint nodes; first[x] becomes the new node's id
__global__ void k_mid_make(const uint32_t* __restrict__ sidx, int64_t n_split,
                           const int32_t* __restrict__ te, const uint64_t* __restrict__ ekey,
                           const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank,
                           int64_t n_nodes, float* __restrict__ xyz, int32_t* __restrict__ first) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 6 * n_split;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[q]) continue;
        const int32_t x = te[6 * (int64_t)sidx[q / 6] + q % 6];
        const uint64_t k = ekey[x];
        const int64_t a = (int64_t)(k >> 32), b = (int64_t)(k & 0xffffffffu);
        const int64_t id = n_nodes + rank[q];
        for (int c = 0; c < 3; ++c)
            xyz[3 * id + c] = (float)(((double)xyz[3 * a + c] + (double)xyz[3 * b + c]) * 0.5);
        first[x] = (int32_t)id;
    }
}

__device__ __forceinline__ double len2(const float* __restrict__ xyz, int i, int j) {
    const double dx = (double)xyz[3 * (int64_t)i] - (double)xyz[3 * (int64_t)j];
    const double dy = (double)xyz[3 * (int64_t)i + 1] - (double)xyz[3 * (int64_t)j + 1];
    const double dz = (double)xyz[3 * (int64_t)i + 2] - (double)xyz[3 * (int64_t)j + 2];
    return dx * dx + dy * dy + dz * dz;
}

// One thread per split tetrahedron r: its 60 edge-slot keys (kEmptyKey where
// the slot meets nothing) and its 8 children's nodes (four corner children,
// then four around the inner octahedron's shortest diagonal, the first of the
// three on ties), appended at n_tets + 8 r.
__global__ void k_events(const uint32_t* __restrict__ sidx, int64_t n_split,
                         const int32_t* __restrict__ te, const int32_t* __restrict__ mid,
                         const int32_t* __restrict__ first, const uint32_t* __restrict__ mflag,
                         const uint64_t* __restrict__ ekey, const float* __restrict__ xyz,
                         int4* __restrict__ tv, int64_t n_tets, uint64_t* __restrict__ evkey) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_split;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = sidx[r];
        const int4 v = tv[t];
        int m[6];
        uint64_t* ev = evkey + 60 * r;
        for (int k = 0; k < 6; ++k) {
            const int32_t x = te[6 * t + k];
            m[k] = mid[x] >= 0 ? mid[x] : first[x];
            if (mflag[6 * r + k]) {
                const uint64_t ab = ekey[x];
                const int a = (int)(ab >> 32), b = (int)(ab & 0xffffffffu);
                ev[2 * k] = key_of(a, m[k]);
                ev[2 * k + 1] = key_of(m[k], b);
            } else {
                ev[2 * k] = ev[2 * k + 1] = kEmptyKey;
            }
        }
        const int m01 = m[0], m02 = m[1], m03 = m[2], m12 = m[3], m13 = m[4], m23 = m[5];
        int4 ch[8];
        ch[0] = make_int4(v.x, m01, m02, m03);
        ch[1] = make_int4(m01, v.y, m12, m13);
        ch[2] = make_int4(m02, m12, v.z, m23);
        ch[3] = make_int4(m03, m13, m23, v.w);
        const int dg[3][2] = {{m01, m23}, {m02, m13}, {m03, m12}};
        const int ring[3][4] = {{m02, m03, m13, m12}, {m01, m03, m23, m12}, {m01, m02, m23, m13}};
        int best = 0;
        double best_l2 = len2(xyz, dg[0][0], dg[0][1]);
        for (int i = 1; i < 3; ++i) {
            const double l2 = len2(xyz, dg[i][0], dg[i][1]);
            if (l2 < best_l2) {
                best = i;
                best_l2 = l2;
            }
        }
        for (int i = 0; i < 4; ++i)
            ch[4 + i] = make_int4(dg[best][0], dg[best][1], ring[best][i], ring[best][(i + 1) & 3]);
        for (int c = 0; c < 8; ++c) {
            tv[n_tets + 8 * r + c] = ch[c];
            for (int e = 0; e < 6; ++e)
                ev[12 + 6 * c + e] = key_of(corner(ch[c], la(e)), corner(ch[c], lb(e)));
        }
    }
}

// evid: the existing edge's id, -1 for an empty slot, -2 pending (new key:
// the smallest slot that meets it is recorded in the level table)
__global__ void k_ev_lookup(const uint64_t* __restrict__ evkey, int64_t n_ev,
                            const uint64_t* __restrict__ hkey, const int32_t* __restrict__ hval,
                            uint64_t hmask, uint64_t* lkey, uint32_t* lslot, uint64_t lmask,
                            int32_t* __restrict__ evid, uint32_t* status) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_ev;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = evkey[q];
        if (k == kEmptyKey) {
            evid[q] = -1;
            continue;
        }
        const int64_t h = table_find(hkey, hmask, k);
        if (h >= 0) {
            evid[q] = hval[h];
            continue;
        }
        evid[q] = -2;
        const int64_t i = table_insert(lkey, lmask, k);
        if (i < 0) atomicOr(status, ST_CAPACITY);
        else atomicMin(lslot + i, (uint32_t)q);
    }
}

__global__ void k_ev_flags(const uint64_t* __restrict__ evkey, const int32_t* __restrict__ evid,
                           int64_t n_ev, const uint64_t* __restrict__ lkey,
                           const uint32_t* __restrict__ lslot, uint64_t lmask,
                           uint32_t* __restrict__ flag) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_ev;
         q += (int64_t)gridDim.x * blockDim.x) {
        bool creator = false;
        if (evid[q] == -2) {
            const int64_t i = table_find(lkey, lmask, evkey[q]);
            creator = i >= 0 && lslot[i] == (uint32_t)q;
        }
        flag[q] = creator ? 1u : 0u;
    }
}

__global__ void k_ev_make(const uint64_t* __restrict__ evkey, const uint32_t* __restrict__ flag,
                          const uint32_t* __restrict__ rank, int64_t n_ev, int64_t n_edges,
                          uint64_t* __restrict__ ekey, int32_t* __restrict__ mid,
                          int2* __restrict__ half, const uint64_t* __restrict__ lkey,
                          int32_t* __restrict__ lid, uint64_t lmask, uint64_t* hkey,
                          int32_t* hval, uint64_t hmask, uint32_t* status) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_ev;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[q]) continue;
        const uint64_t k = evkey[q];
        const int32_t id = (int32_t)(n_edges + rank[q]);
        ekey[id] = k;
        mid[id] = -1;
        half[id] = make_int2(-1, -1);
        const int64_t i = table_find(lkey, lmask, k);
        if (i >= 0) lid[i] = id;
        const int64_t h = table_insert(hkey, hmask, k);
        if (h < 0) atomicOr(status, ST_CAPACITY);
        else hval[h] = id;
    }
}

__global__ void k_ev_resolve(const uint64_t* __restrict__ evkey, int32_t* __restrict__ evid,
                             int64_t n_ev, const uint64_t* __restrict__ lkey,
                             const int32_t* __restrict__ lid, uint64_t lmask) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_ev;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (evid[q] != -2) continue;
        const int64_t i = table_find(lkey, lmask, evkey[q]);
        evid[q] = i >= 0 ? lid[i] : -1;
    }
}

// The children's edges, depth and leaf flags; the parent stops being a leaf;
// the edges split here get their midpoints and halves.
__global__ void k_kids(const uint32_t* __restrict__ sidx, int64_t n_split,
                       const int32_t* __restrict__ evid, int64_t n_tets,
                       int32_t* __restrict__ te, int32_t* __restrict__ depth,
                       uint8_t* __restrict__ leaf, const uint32_t* __restrict__ mflag,
                       const int32_t* __restrict__ first, int32_t* __restrict__ mid,
                       int2* __restrict__ half) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_split;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = sidx[r];
        const int32_t* ev = evid + 60 * r;
        const int32_t d = depth[t] + 1;
        for (int c = 0; c < 8; ++c) {
            const int64_t id = n_tets + 8 * r + c;
            for (int e = 0; e < 6; ++e) te[6 * id + e] = ev[12 + 6 * c + e];
            depth[id] = d;
            leaf[id] = 1;
        }
        leaf[t] = 0;
        for (int k = 0; k < 6; ++k) {
            if (!mflag[6 * r + k]) continue;
            const int32_t x = te[6 * t + k];
            half[x] = make_int2(ev[2 * k], ev[2 * k + 1]);
            mid[x] = first[x];
        }
    }
}

// ---- the final lattice ----

__global__ void k_seg_flags(const int2* __restrict__ half, int64_t n, uint32_t* __restrict__ f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = half[i].x < 0 ? 1u : 0u;
}

__global__ void k_leaf_flags(const uint8_t* __restrict__ leaf, int64_t n, uint32_t* __restrict__ f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = leaf[i] ? 1u : 0u;
}

// Positive floats order as their bit patterns: atomicMin on the bits.
__global__ void k_edge_min(const uint32_t* __restrict__ leaves, int64_t n_leaf,
                           const int32_t* __restrict__ te, const int2* __restrict__ half,
                           const uint32_t* __restrict__ seg_of, const float* __restrict__ ratio,
                           uint32_t* __restrict__ bits, uint32_t* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_leaf;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = leaves[i];
        const uint32_t rb = __float_as_uint(ratio[t]);
        for (int e = 0; e < 6; ++e) {
            int32_t stack[40];
            int sp = 0;
            stack[sp++] = te[6 * t + e];
            while (sp > 0) {
                const int32_t x = stack[--sp];
                const int2 h = half[x];
                if (h.x < 0) {
                    atomicMin(bits + seg_of[x], rb);
                } else if (sp + 2 <= 40) {
                    stack[sp++] = h.y;
                    stack[sp++] = h.x;
                } else {
                    atomicOr(status, ST_CAPACITY);
                }
            }
        }
    }
}

__global__ void k_seg_points(const uint32_t* __restrict__ segs, int64_t n,
                             const uint64_t* __restrict__ ekey, const float* __restrict__ xyz,
                             float4* __restrict__ sa, float4* __restrict__ sb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ekey[segs[i]];
        const int64_t a = (int64_t)(k >> 32), b = (int64_t)(k & 0xffffffffu);
        sa[i] = make_float4(xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2], 0.0f);
        sb[i] = make_float4(xyz[3 * b], xyz[3 * b + 1], xyz[3 * b + 2], 0.0f);
    }
}

__global__ void k_gather_edges(const uint32_t* __restrict__ segs, int64_t n,
                               const uint64_t* __restrict__ ekey, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ekey[segs[i]];
        out[2 * i] = (int32_t)(k >> 32);
        out[2 * i + 1] = (int32_t)(k & 0xffffffffu);
    }
}

__global__ void k_gather_leaves(const uint32_t* __restrict__ leaves, int64_t n,
                                const int4* __restrict__ tv, const int32_t* __restrict__ tdepth,
                                const double* __restrict__ t_target, const float* __restrict__ t_rho,
                                const float* __restrict__ t_ratio, int4* __restrict__ tets,
                                int32_t* __restrict__ depth, double* __restrict__ target,
                                float* __restrict__ rho, float* __restrict__ ratio) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = leaves[i];
        tets[i] = tv[t];
        depth[i] = tdepth[t];
        target[i] = t_target[t];
        rho[i] = t_rho[t];
        ratio[i] = t_ratio[t];
    }
}

// Grows b to at least `need` bytes keeping its first `used` bytes.
void grow(DevBuf& b, size_t used, size_t need, cudaStream_t s) {
    if (need <= b.size()) return;
    DevBuf nb(std::max(need, b.size() + b.size() / 2), s);
    if (used) CSL_CUDA(cudaMemcpyAsync(nb.get(), b.get(), used, cudaMemcpyDeviceToDevice, s));
    b = std::move(nb);
}

uint64_t pow2_at_least(uint64_t n) {
    uint64_t c = 64;
    while (c < n) c <<= 1;
    return c;
}

void rebuild_hash(DevMesh& m, uint64_t cap, cudaStream_t s) {
    m.hkey.alloc((size_t)cap * 8, s);
    m.hval.alloc((size_t)cap * 4, s);
    m.hcap = (int64_t)cap;
    CSL_CUDA(cudaMemsetAsync(m.hkey.get(), 0xff, (size_t)cap * 8, s));
    if (m.n_edges > 0) {
        k_hash_build<<<grid_for(m.n_edges, 256), 256, 0, s>>>(
            m.ekey.as<uint64_t>(), m.n_edges, m.hkey.as<uint64_t>(), m.hval.as<int32_t>(),
            cap - 1, m.status.as<uint32_t>());
        CSL_LAUNCH_CHECK("edge table");
    }
}

void check_status(const DevMesh& m, cudaStream_t s) {
    uint32_t st = 0;
    read_to_host(&st, m.status.get(), 4, s);
    if (st) fail(CSL_ERR_CAPACITY, "density matching: an edge table or a segment walk ran full");
}

}  // namespace

void mesh_init(DevMesh& m, const float* nodes, int64_t n_nodes, const int32_t* tets,
               int64_t n_tets, cudaStream_t s) {
    m.n_nodes = n_nodes;
    m.n_tets = n_tets;
    m.status.alloc(4, s);
    CSL_CUDA(cudaMemsetAsync(m.status.get(), 0, 4, s));
    m.xyz.alloc((size_t)std::max<int64_t>(n_nodes, 1) * 12, s);
    if (n_nodes)
        CSL_CUDA(cudaMemcpyAsync(m.xyz.get(), nodes, (size_t)n_nodes * 12, cudaMemcpyHostToDevice, s));
    m.tv.alloc((size_t)std::max<int64_t>(n_tets, 1) * 16, s);
    m.te.alloc((size_t)std::max<int64_t>(n_tets, 1) * 24, s);
    m.depth.alloc((size_t)std::max<int64_t>(n_tets, 1) * 4, s);
    m.leaf.alloc((size_t)std::max<int64_t>(n_tets, 1), s);
    const int64_t n_ev = 6 * n_tets;
    if (n_tets) {
        CSL_CUDA(cudaMemcpyAsync(m.tv.get(), tets, (size_t)n_tets * 16, cudaMemcpyHostToDevice, s));
        CSL_CUDA(cudaMemsetAsync(m.depth.get(), 0, (size_t)n_tets * 4, s));
        CSL_CUDA(cudaMemsetAsync(m.leaf.get(), 1, (size_t)n_tets, s));
    }
    m.n_edges = 0;
    if (n_ev > 0) {
        // the input's edges in (smaller, larger) node order: a stable sort by
        // the larger node, then by the smaller one; a run of equal keys is one edge
        DevBuf k((size_t)n_ev * 4, s), v((size_t)n_ev * 4, s), tk((size_t)n_ev * 4, s),
            tvb((size_t)n_ev * 4, s), rank((size_t)n_ev * 4, s), tot(8, s);
        int bits = 1;
        while (bits < 32 && ((int64_t)1 << bits) < n_nodes) ++bits;
        const unsigned g = grid_for(n_ev, 256);
        k_init_events<<<g, 256, 0, s>>>(m.tv.as<int4>(), n_tets, k.as<uint32_t>(), v.as<uint32_t>());
        CSL_LAUNCH_CHECK("mesh events");
        radix_sort_pairs(k.as<uint32_t>(), v.as<uint32_t>(), tk.as<uint32_t>(), tvb.as<uint32_t>(),
                         n_ev, bits, s);
        k_init_key2<<<g, 256, 0, s>>>(m.tv.as<int4>(), v.as<uint32_t>(), n_ev, k.as<uint32_t>());
        CSL_LAUNCH_CHECK("mesh second key");
        radix_sort_pairs(k.as<uint32_t>(), v.as<uint32_t>(), tk.as<uint32_t>(), tvb.as<uint32_t>(),
                         n_ev, bits, s);
        k_init_unique<<<g, 256, 0, s>>>(m.tv.as<int4>(), v.as<uint32_t>(), n_ev, k.as<uint32_t>());
        CSL_LAUNCH_CHECK("mesh unique edges");
        exclusive_scan_u32(k.as<uint32_t>(), rank.as<uint32_t>(), n_ev, tot.as<uint32_t>(), s);
        uint32_t ne = 0;
        read_to_host(&ne, tot.get(), 4, s);
        m.n_edges = ne;
        m.ekey.alloc((size_t)std::max<int64_t>(ne, 1) * 8, s);
        k_init_edges<<<g, 256, 0, s>>>(m.tv.as<int4>(), v.as<uint32_t>(), k.as<uint32_t>(),
                                       rank.as<uint32_t>(), n_ev, m.ekey.as<uint64_t>(),
                                       m.te.as<int32_t>());
        CSL_LAUNCH_CHECK("mesh edges");
    } else {
        m.ekey.alloc(8, s);
    }
    m.mid.alloc((size_t)std::max<int64_t>(m.n_edges, 1) * 4, s);
    m.half.alloc((size_t)std::max<int64_t>(m.n_edges, 1) * 8, s);
    if (m.n_edges) {
        CSL_CUDA(cudaMemsetAsync(m.mid.get(), 0xff, (size_t)m.n_edges * 4, s));
        CSL_CUDA(cudaMemsetAsync(m.half.get(), 0xff, (size_t)m.n_edges * 8, s));
    }
    rebuild_hash(m, pow2_at_least(2 * (uint64_t)std::max<int64_t>(m.n_edges, 1)), s);
}

void mesh_corners(const DevMesh& m, int64_t t0, int64_t n, float4* out, cudaStream_t s) {
    if (n <= 0) return;
    k_corners<<<grid_for(4 * n, 256), 256, 0, s>>>(m.tv.as<int4>(), m.xyz.as<float>(), t0, n, out);
    CSL_LAUNCH_CHECK("tetrahedron corners");
}

int64_t mesh_subdivide(DevMesh& m, int64_t t0, int64_t n, const uint32_t* split, cudaStream_t s) {
    if (n <= 0) return 0;
    DevBuf rank((size_t)n * 4, s), cnt(16, s);
    CSL_CUDA(cudaMemsetAsync(cnt.get(), 0, 16, s));
    uint32_t* c = cnt.as<uint32_t>();
    exclusive_scan_u32(split, rank.as<uint32_t>(), n, c, s);
    uint32_t ns32 = 0;
    read_to_host(&ns32, c, 4, s);
    const int64_t ns = ns32;
    if (ns == 0) return 0;
    if (m.n_tets + 8 * ns >= ((int64_t)1 << 27)) fail(CSL_ERR_CAPACITY, "more than 2^27 tetrahedra");
    if (m.n_edges + 60 * ns >= ((int64_t)1 << 31) || m.n_nodes + 6 * ns >= ((int64_t)1 << 30))
        fail(CSL_ERR_CAPACITY, "too many nodes or edges");
    DevBuf sidx((size_t)ns * 4, s);
    k_list<<<grid_for(n, 256), 256, 0, s>>>(split, rank.as<uint32_t>(), n, t0, sidx.as<uint32_t>());
    CSL_LAUNCH_CHECK("split list");

    // room for the level's new items
    const int64_t nt = m.n_tets + 8 * ns, nn_max = m.n_nodes + 6 * ns, ne_max = m.n_edges + 60 * ns;
    grow(m.tv, (size_t)m.n_tets * 16, (size_t)nt * 16, s);
    grow(m.te, (size_t)m.n_tets * 24, (size_t)nt * 24, s);
    grow(m.depth, (size_t)m.n_tets * 4, (size_t)nt * 4, s);
    grow(m.leaf, (size_t)m.n_tets, (size_t)nt, s);
    grow(m.xyz, (size_t)m.n_nodes * 12, (size_t)nn_max * 12, s);
    grow(m.ekey, (size_t)m.n_edges * 8, (size_t)ne_max * 8, s);
    grow(m.mid, (size_t)m.n_edges * 4, (size_t)ne_max * 4, s);
    grow(m.half, (size_t)m.n_edges * 8, (size_t)ne_max * 8, s);
    if ((uint64_t)m.hcap < 2 * (uint64_t)ne_max) rebuild_hash(m, pow2_at_least(2 * (uint64_t)ne_max), s);

    // midpoints
    const int64_t n6 = 6 * ns, n60 = 60 * ns;
    DevBuf first((size_t)m.n_edges * 4, s), mflag((size_t)n6 * 4, s), mrank((size_t)n6 * 4, s);
    CSL_CUDA(cudaMemsetAsync(first.get(), 0x7f, (size_t)m.n_edges * 4, s));
    const unsigned g6 = grid_for(n6, 256), g60 = grid_for(n60, 256), g1 = grid_for(ns, 128);
    k_mid_claim<<<g6, 256, 0, s>>>(sidx.as<uint32_t>(), ns, m.te.as<int32_t>(), m.mid.as<int32_t>(),
                                   first.as<int32_t>());
    CSL_LAUNCH_CHECK("midpoint claims");
    k_mid_flags<<<g6, 256, 0, s>>>(sidx.as<uint32_t>(), ns, m.te.as<int32_t>(), m.mid.as<int32_t>(),
                                   first.as<int32_t>(), mflag.as<uint32_t>());
    CSL_LAUNCH_CHECK("midpoint creators");
    exclusive_scan_u32(mflag.as<uint32_t>(), mrank.as<uint32_t>(), n6, c + 1, s);
    k_mid_make<<<g6, 256, 0, s>>>(sidx.as<uint32_t>(), ns, m.te.as<int32_t>(), m.ekey.as<uint64_t>(),
                                  mflag.as<uint32_t>(), mrank.as<uint32_t>(), m.n_nodes,
                                  m.xyz.as<float>(), first.as<int32_t>());
    CSL_LAUNCH_CHECK("midpoints");

    // edges: the slots' keys, existing edges, the first slot of every new key
    DevBuf evkey((size_t)n60 * 8, s), evid((size_t)n60 * 4, s), eflag((size_t)n60 * 4, s),
        erank((size_t)n60 * 4, s);
    const uint64_t lcap = pow2_at_least(2 * (uint64_t)n60);
    DevBuf lkey((size_t)lcap * 8, s), lslot((size_t)lcap * 4, s), lid((size_t)lcap * 4, s);
    CSL_CUDA(cudaMemsetAsync(lkey.get(), 0xff, (size_t)lcap * 8, s));
    CSL_CUDA(cudaMemsetAsync(lslot.get(), 0xff, (size_t)lcap * 4, s));
    k_events<<<g1, 128, 0, s>>>(sidx.as<uint32_t>(), ns, m.te.as<int32_t>(), m.mid.as<int32_t>(),
                                first.as<int32_t>(), mflag.as<uint32_t>(), m.ekey.as<uint64_t>(),
                                m.xyz.as<float>(), m.tv.as<int4>(), m.n_tets,
                                evkey.as<uint64_t>());
    CSL_LAUNCH_CHECK("subdivision slots");
    const uint64_t hmask = (uint64_t)m.hcap - 1, lmask = lcap - 1;
    k_ev_lookup<<<g60, 256, 0, s>>>(evkey.as<uint64_t>(), n60, m.hkey.as<uint64_t>(),
                                    m.hval.as<int32_t>(), hmask, lkey.as<uint64_t>(),
                                    lslot.as<uint32_t>(), lmask, evid.as<int32_t>(),
                                    m.status.as<uint32_t>());
    CSL_LAUNCH_CHECK("edge lookups");
    k_ev_flags<<<g60, 256, 0, s>>>(evkey.as<uint64_t>(), evid.as<int32_t>(), n60,
                                   lkey.as<uint64_t>(), lslot.as<uint32_t>(), lmask,
                                   eflag.as<uint32_t>());
    CSL_LAUNCH_CHECK("edge creators");
    exclusive_scan_u32(eflag.as<uint32_t>(), erank.as<uint32_t>(), n60, c + 2, s);
    k_ev_make<<<g60, 256, 0, s>>>(evkey.as<uint64_t>(), eflag.as<uint32_t>(), erank.as<uint32_t>(),
                                  n60, m.n_edges, m.ekey.as<uint64_t>(), m.mid.as<int32_t>(),
                                  m.half.as<int2>(), lkey.as<uint64_t>(), lid.as<int32_t>(), lmask,
                                  m.hkey.as<uint64_t>(), m.hval.as<int32_t>(), hmask,
                                  m.status.as<uint32_t>());
    CSL_LAUNCH_CHECK("new edges");
    k_ev_resolve<<<g60, 256, 0, s>>>(evkey.as<uint64_t>(), evid.as<int32_t>(), n60,
                                     lkey.as<uint64_t>(), lid.as<int32_t>(), lmask);
    CSL_LAUNCH_CHECK("edge ids");
    k_kids<<<g1, 128, 0, s>>>(sidx.as<uint32_t>(), ns, evid.as<int32_t>(), m.n_tets,
                              m.te.as<int32_t>(), m.depth.as<int32_t>(), m.leaf.as<uint8_t>(),
                              mflag.as<uint32_t>(), first.as<int32_t>(), m.mid.as<int32_t>(),
                              m.half.as<int2>());
    CSL_LAUNCH_CHECK("children");
    uint32_t counts[4];
    read_to_host(counts, c, 16, s);
    check_status(m, s);
    m.n_nodes += counts[1];
    m.n_edges += counts[2];
    m.n_tets = nt;
    return ns;
}

void mesh_finalize(const DevMesh& m, MeshFinal& f, cudaStream_t s) {
    DevBuf cnt(8, s);
    CSL_CUDA(cudaMemsetAsync(cnt.get(), 0, 8, s));
    uint32_t* c = cnt.as<uint32_t>();
    {
        const int64_t n = m.n_edges;
        DevBuf flag((size_t)std::max<int64_t>(n, 1) * 4, s);
        f.seg_of.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
        if (n) {
            k_seg_flags<<<grid_for(n, 256), 256, 0, s>>>(m.half.as<int2>(), n, flag.as<uint32_t>());
            CSL_LAUNCH_CHECK("segment flags");
        }
        exclusive_scan_u32(flag.as<uint32_t>(), f.seg_of.as<uint32_t>(), n, c, s);
        uint32_t ns = 0;
        read_to_host(&ns, c, 4, s);
        f.n_seg = ns;
        f.segs.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
        if (n) {
            k_list<<<grid_for(n, 256), 256, 0, s>>>(flag.as<uint32_t>(), f.seg_of.as<uint32_t>(), n,
                                                    0, f.segs.as<uint32_t>());
            CSL_LAUNCH_CHECK("segments");
        }
    }
    {
        const int64_t n = m.n_tets;
        DevBuf flag((size_t)std::max<int64_t>(n, 1) * 4, s), rank((size_t)std::max<int64_t>(n, 1) * 4, s);
        if (n) {
            k_leaf_flags<<<grid_for(n, 256), 256, 0, s>>>(m.leaf.as<uint8_t>(), n, flag.as<uint32_t>());
            CSL_LAUNCH_CHECK("leaf flags");
        }
        exclusive_scan_u32(flag.as<uint32_t>(), rank.as<uint32_t>(), n, c + 1, s);
        uint32_t nl = 0;
        read_to_host(&nl, c + 1, 4, s);
        f.n_leaf = nl;
        f.leaves.alloc((size_t)std::max<int64_t>(nl, 1) * 4, s);
        if (n) {
            k_list<<<grid_for(n, 256), 256, 0, s>>>(flag.as<uint32_t>(), rank.as<uint32_t>(), n, 0,
                                                    f.leaves.as<uint32_t>());
            CSL_LAUNCH_CHECK("leaves");
        }
    }
}

void mesh_edge_min(const DevMesh& m, const MeshFinal& f, const float* tet_ratio,
                   uint32_t* ratio_bits, cudaStream_t s) {
    if (f.n_leaf <= 0) return;
    k_edge_min<<<grid_for(f.n_leaf, 256), 256, 0, s>>>(
        f.leaves.as<uint32_t>(), f.n_leaf, m.te.as<int32_t>(), m.half.as<int2>(),
        f.seg_of.as<uint32_t>(), tet_ratio, ratio_bits, m.status.as<uint32_t>());
    CSL_LAUNCH_CHECK("edge ratio minimum");
    check_status(m, s);
}

void mesh_segment_points(const DevMesh& m, const MeshFinal& f, float4* sa, float4* sb,
                         cudaStream_t s) {
    if (f.n_seg <= 0) return;
    k_seg_points<<<grid_for(f.n_seg, 256), 256, 0, s>>>(f.segs.as<uint32_t>(), f.n_seg,
                                                        m.ekey.as<uint64_t>(), m.xyz.as<float>(),
                                                        sa, sb);
    CSL_LAUNCH_CHECK("segment points");
}

void mesh_gather_final(const DevMesh& m, const MeshFinal& f, int32_t* edges, int32_t* tets,
                       int32_t* depth, const double* t_target, double* target,
                       const float* t_rho, float* rho, const float* t_ratio, float* ratio,
                       cudaStream_t s) {
    if (f.n_seg > 0) {
        k_gather_edges<<<grid_for(f.n_seg, 256), 256, 0, s>>>(f.segs.as<uint32_t>(), f.n_seg,
                                                              m.ekey.as<uint64_t>(), edges);
        CSL_LAUNCH_CHECK("segment nodes");
    }
    if (f.n_leaf > 0) {
        k_gather_leaves<<<grid_for(f.n_leaf, 256), 256, 0, s>>>(
            f.leaves.as<uint32_t>(), f.n_leaf, m.tv.as<int4>(), m.depth.as<int32_t>(), t_target,
            t_rho, t_ratio, reinterpret_cast<int4*>(tets), depth, target, rho, ratio);
        CSL_LAUNCH_CHECK("leaves' values");
    }
}

}  // namespace csl
