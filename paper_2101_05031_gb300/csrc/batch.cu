// Batched slicing: many (lattice, slicing request) jobs as one CUDA graph.
//
// Planning runs every job once through the ordinary pipeline (binner, field,
// contours), recording the sizes that each stage discovers and keeping every
// output buffer at those sizes. The graph is a capture of the replay of all
// jobs, which reads nothing back: the binner and contour stages of the jobs
// run on parallel branches (round-robin over a few streams), and the field of
// all jobs is one persistent kernel over a (job, slab, tile) queue sorted
// longest tile list first. Every size that the device finds is checked
// against the plan; a mismatch sets a device flag (copied to pinned host
// memory by the graph's last node) and bounds every write.
//
// The autotuner times the whole graph for each slab depth and persistent
// grid size and keeps the fastest; the choice is cached per process under a
// hash of the job sizes.
#include <string.h>

#include <chrono>
#include <functional>
#include <map>
#include <mutex>
#include <new>

#include "slice.cuh"

using namespace csl;

struct csl_batch {
    struct Job {
        csl_lattice* L = nullptr;
        csl_slice_desc d{};
        ChunkGeom g{};
        ChunkPlan plan;
        SlabBins bins;
        ChunkContours cont;
        float* sigma = nullptr;
        uint32_t* mask = nullptr;
        int64_t mask_words = 0;
        bool want_eid = false;
    };
    std::vector<Job> jobs;
    int S = 8, ctas = 4, n_sm = 0, branches = 8;
    int kernel = CSL_FIELD_BLOCK, T = 16, K = 256;   // field kernel, tile, staging chunk
    cudaStream_t st = nullptr;           // planning, capture and copies
    std::vector<cudaStream_t> side;      // capture branches
    std::vector<cudaEvent_t> ev;         // fork / join events of the capture
    DevBuf sigma_arena, mask_arena, flag_d;
    int64_t mask_arena_words = 0;
    uint32_t* flag_h = nullptr;          // pinned
    FieldBatch fb;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    csl_batch_info info{};

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~csl_batch() {
        if (st) cudaStreamSynchronize(st);
        drop_graph();
        fb = FieldBatch();
        jobs.clear();   // stream-ordered buffers are freed on st
        sigma_arena.release();
        mask_arena.release();
        flag_d.release();
        if (st) cudaStreamSynchronize(st);
        if (flag_h) cudaFreeHost(flag_h);
        for (auto e : ev) cudaEventDestroy(e);
        for (auto s : side) cudaStreamDestroy(s);
        if (st) cudaStreamDestroy(st);
        cudaGetLastError();
    }
};

namespace {

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

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---- per-process autotuning cache ----
std::mutex& g_tune_cache_mu() {
    static std::mutex mu;
    return mu;
}
// key -> (slab, CTAs per SM, field kernel, tile, staging chunk)
struct TuneChoice {
    int S, ctas, kernel, T, K;
};
std::map<uint64_t, TuneChoice> g_tune_cache;

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

uint64_t workload_key(const csl_batch* b) {
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &dev, sizeof dev);
    h = fnv(h, &b->n_sm, sizeof b->n_sm);
    const size_t n = b->jobs.size();
    h = fnv(h, &n, sizeof n);
    for (const auto& J : b->jobs) {
        const int64_t v[5] = {J.L->n_edges, J.L->n_nodes, J.d.nx, J.d.ny, J.d.n_layers};
        const double w[3] = {J.d.pixel, J.d.dz, J.L->R};
        h = fnv(h, v, sizeof v);
        h = fnv(h, w, sizeof w);
    }
    return h;
}

// ---- planning: every job once through the ordinary (reading) pipeline ----
void plan_jobs(csl_batch* b, int S, int kernel, int T, int K) {
    b->drop_graph();
    b->fb = FieldBatch();
    uint32_t* flag = b->flag_d.as<uint32_t>();
    CSL_CUDA(cudaMemsetAsync(flag, 0, 4, b->st));
    for (auto& J : b->jobs) {
        csl_slice_desc d = J.d;
        d.slab = S;
        d.tile = T;
        d.field_kernel = (int16_t)kernel;
        d.stage_records = (int16_t)K;
        d.flags &= ~CSL_SLICE_FUSED;
        d.chunk_layers = d.n_layers;
        const SlicePlan p = make_plan(J.L, d);
        require_arg(p.chunk >= d.n_layers,
                    "batch: a job must fit one chunk (fewer than 2^27 contour edge words)");
        J.g = chunk_geom(J.L, d, p, 0, d.n_layers);
        J.plan = ChunkPlan();
        J.bins = SlabBins();
        J.cont = ChunkContours();
        Replay rp{false, &J.plan, flag};
        bin_chunk(J.L, J.g, J.bins, b->st, &rp);
    }
    CSL_CUDA(cudaMemsetAsync(b->mask_arena.get(), 0, (size_t)b->mask_arena_words * 4, b->st));
    std::vector<FieldBatchJob> fj;
    for (auto& J : b->jobs)
        fj.push_back(FieldBatchJob{J.L, J.g, &J.bins, J.sigma, J.mask, b->flag_d.as<uint32_t>()});
    field_batch_prepare(fj, b->fb, b->st);
    field_batch_run(b->fb, b->n_sm * b->ctas, b->st);
    for (auto& J : b->jobs) {
        Replay rp{false, &J.plan, flag};
        contours_chunk(J.g, J.L->C, J.sigma, J.mask, J.want_eid, J.cont, b->st, &rp);
    }
    uint32_t f = 0;
    read_to_host(&f, flag, 4, b->st);
    if (f) fail(CSL_ERR_CUDA, "batch planning: a stage reported inconsistent sizes");
    b->S = S;
    b->kernel = kernel;
    b->T = T;
    b->K = K;
    int64_t pairs = 0, cross = 0, loops = 0;
    for (auto& J : b->jobs) {
        pairs += J.plan.n_pairs;
        cross += J.plan.n_cross;
        loops += J.plan.n_loops;
    }
    b->info.n_pairs = pairs;
    b->info.n_crossings = cross;
    b->info.n_loops = loops;
    b->info.n_items = b->fb.n_items;
}

// ---- capture of the replay ----
void fork(csl_batch* b, int base) {
    CSL_CUDA(cudaEventRecord(b->ev[base], b->st));
    for (auto s : b->side) CSL_CUDA(cudaStreamWaitEvent(s, b->ev[base], 0));
}

void join(csl_batch* b, int base) {
    for (size_t k = 0; k < b->side.size(); ++k) {
        CSL_CUDA(cudaEventRecord(b->ev[base + 1 + k], b->side[k]));
        CSL_CUDA(cudaStreamWaitEvent(b->st, b->ev[base + 1 + k], 0));
    }
}

void capture(csl_batch* b, int ctas) {
    b->drop_graph();
    const int K = (int)b->side.size();
    uint32_t* flag = b->flag_d.as<uint32_t>();
    CSL_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    try {
        CSL_CUDA(cudaMemsetAsync(flag, 0, 4, b->st));
        fork(b, 0);
        for (size_t j = 0; j < b->jobs.size(); ++j) {
            auto& J = b->jobs[j];
            Replay rp{true, &J.plan, flag};
            bin_chunk(J.L, J.g, J.bins, b->side[j % K], &rp);
        }
        join(b, 0);
        CSL_CUDA(cudaMemsetAsync(b->mask_arena.get(), 0, (size_t)b->mask_arena_words * 4, b->st));
        field_batch_run(b->fb, b->n_sm * ctas, b->st);
        fork(b, K + 1);
        for (size_t j = 0; j < b->jobs.size(); ++j) {
            auto& J = b->jobs[j];
            Replay rp{true, &J.plan, flag};
            contours_chunk(J.g, J.L->C, J.sigma, J.mask, J.want_eid, J.cont, b->side[j % K],
                           &rp);
        }
        join(b, K + 1);
        CSL_CUDA(cudaMemcpyAsync(b->flag_h, flag, 4, cudaMemcpyDeviceToHost, b->st));
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->st, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    CSL_CUDA(cudaStreamEndCapture(b->st, &b->graph));
    CSL_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    size_t n = 0;
    CSL_CUDA(cudaGraphGetNodes(b->graph, nullptr, &n));
    b->info.graph_nodes = (int64_t)n;
    b->ctas = ctas;
}

void launch_and_check(csl_batch* b, cudaStream_t s) {
    *b->flag_h = 0xffffffffu;
    CSL_CUDA(cudaGraphLaunch(b->exec, s));
    CSL_CUDA(cudaStreamSynchronize(s));
    const uint32_t f = *b->flag_h;
    if (f == 0xffffffffu) fail(CSL_ERR_CUDA, "batch: the graph did not report its status");
    if (f)
        fail(CSL_ERR_CAPACITY,
             "batch: the device found sizes other than the plan's (inputs changed); "
             "create the batch again");
}

// Best of two timed launches after one untimed one (ms).
float time_graph(csl_batch* b) {
    launch_and_check(b, b->st);
    cudaEvent_t e0, e1;
    CSL_CUDA(cudaEventCreate(&e0));
    CSL_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < 2; ++r) {
        CSL_CUDA(cudaEventRecord(e0, b->st));
        CSL_CUDA(cudaGraphLaunch(b->exec, b->st));
        CSL_CUDA(cudaEventRecord(e1, b->st));
        CSL_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CSL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (*b->flag_h) fail(CSL_ERR_CUDA, "batch: a tuning run reported inconsistent sizes");
    return best;
}

const csl_batch::Job& job_at(const csl_batch* b, int32_t j) {
    require_arg(b != nullptr, "batch is NULL");
    require_arg(j >= 0 && j < (int32_t)b->jobs.size(), "job index out of range");
    return b->jobs[j];
}

}  // namespace

extern "C" {

csl_status csl_batch_create(csl_lattice* const* lats, const csl_slice_desc* descs, int32_t n_jobs,
                            const csl_batch_opts* opts, void* stream, csl_batch** out) {
    return guard([&] {
        require_arg(out != nullptr, "out is NULL");
        *out = nullptr;
        require_arg(n_jobs >= 1, "n_jobs must be >= 1");
        require_arg(lats != nullptr && descs != nullptr, "lats or descs is NULL");
        csl_batch_opts o = {0, 0, 0, 0, 0, 0, 0, 0};
        if (opts) o = *opts;
        require_arg(o.field_kernel == CSL_FIELD_AUTO || o.field_kernel == CSL_FIELD_BLOCK ||
                        o.field_kernel == CSL_FIELD_FOOTPRINT,
                    "field_kernel must be CSL_FIELD_AUTO, CSL_FIELD_BLOCK or CSL_FIELD_FOOTPRINT");
        require_arg(o.tile == 0 || o.tile == 16 || o.tile == 32, "tile must be 0, 16 or 32");
        require_arg(o.tile != 32 || o.field_kernel == CSL_FIELD_FOOTPRINT,
                    "32-pixel tiles need the footprint field kernel");
        require_arg(o.stage_records == 0 || (o.stage_records >= 32 && o.stage_records <= 1024 &&
                                             o.stage_records % 32 == 0),
                    "stage_records must be 0 or a multiple of 32 up to 1024");
        require_arg(o.slab == 0 || o.slab == 2 || o.slab == 4 || o.slab == 8,
                    "slab must be 0, 2, 4 or 8");
        require_arg(o.ctas_per_sm >= 0 && o.ctas_per_sm <= 6, "ctas_per_sm must be in [0, 6]");
        require_arg(o.branches >= 0 && o.branches <= 32, "branches must be in [0, 32]");
        cudaStream_t user = (cudaStream_t)stream;
        CSL_CUDA(cudaStreamSynchronize(user));   // inputs enqueued before the call are ready

        csl_batch* b = new csl_batch();
        try {
            int dev = 0;
            CSL_CUDA(cudaGetDevice(&dev));
            CSL_CUDA(cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev));
            CSL_CUDA(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
            b->branches = o.branches ? o.branches : 8;
            b->branches = std::min<int>(b->branches, n_jobs);
            b->side.resize(b->branches, nullptr);
            for (auto& s : b->side) CSL_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            b->ev.resize(2 * (b->branches + 1), nullptr);
            for (auto& e : b->ev)
                CSL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            CSL_CUDA(cudaHostAlloc((void**)&b->flag_h, 4, cudaHostAllocDefault));
            b->flag_d.alloc_persistent(4);

            int min_layers = 1 << 30;
            int64_t sigma_floats = 0, mask_words = 0;
            b->jobs.resize(n_jobs);
            for (int j = 0; j < n_jobs; ++j) {
                auto& J = b->jobs[j];
                require_arg(lats[j] != nullptr, "a job's lattice is NULL");
                require_device_resident(lats[j]);
                validate_desc(&descs[j]);
                require_arg(descs[j].n_layers >= 1, "a batch job needs n_layers >= 1");
                J.L = lats[j];
                J.d = descs[j];
                J.d.sigma_out = nullptr;
                J.d.mask_out = nullptr;
                J.want_eid = (J.d.flags & CSL_SLICE_EDGE_IDS) != 0;
                min_layers = std::min(min_layers, J.d.n_layers);
                sigma_floats += (int64_t)J.d.n_layers * J.d.nx * J.d.ny;
                J.mask_words = (int64_t)J.d.n_layers * mask_words_per_layer(J.d.nx, J.d.ny);
                mask_words += J.mask_words;
            }
            b->info.n_jobs = n_jobs;
            b->info.pixel_evals = sigma_floats;
            b->sigma_arena.alloc_persistent((size_t)sigma_floats * 4);
            b->mask_arena.alloc_persistent((size_t)mask_words * 4);
            b->mask_arena_words = mask_words;
            int64_t so = 0, mo = 0;
            for (auto& J : b->jobs) {
                J.sigma = b->sigma_arena.as<float>() + so;
                J.mask = b->mask_arena.as<uint32_t>() + mo;
                so += (int64_t)J.d.n_layers * J.d.nx * J.d.ny;
                mo += J.mask_words;
            }

            const int S0 = min_layers >= 8 ? 8 : (min_layers >= 4 ? 4 : 2);
            int S = o.slab ? o.slab : S0;
            int ctas = o.ctas_per_sm ? o.ctas_per_sm : 4;
            int kernel = o.field_kernel == CSL_FIELD_FOOTPRINT ? CSL_FIELD_FOOTPRINT
                                                               : CSL_FIELD_BLOCK;
            int T = o.tile ? o.tile : (kernel == CSL_FIELD_FOOTPRINT ? 32 : 16);
            int K = o.stage_records ? o.stage_records : 256;
            const uint64_t key = workload_key(b);
            bool tune = o.autotune != 0;
            if (tune) {
                std::lock_guard<std::mutex> lk(g_tune_cache_mu());
                auto it = g_tune_cache.find(key);
                if (it != g_tune_cache.end()) {
                    S = it->second.S;
                    ctas = it->second.ctas;
                    kernel = it->second.kernel;
                    T = it->second.T;
                    K = it->second.K;
                    tune = false;
                    b->info.from_cache = 1;
                }
            }
            if (tune) {
                const double t0 = now_ms();
                double plan_ms = 0.0;
                float best = 1e30f;
                TuneChoice bc{S0, 4, CSL_FIELD_BLOCK, 16, 256};
                int nc = 0;
                auto plan = [&](int s_, int k_, int t_, int K_) {
                    if (b->S == s_ && b->kernel == k_ && b->T == t_ && b->K == K_ && b->fb.n_items)
                        return;
                    const double tp = now_ms();
                    plan_jobs(b, s_, k_, t_, K_);
                    plan_ms += now_ms() - tp;
                };
                auto try_one = [&](int s_, int c_, int k_, int t_, int K_) {
                    plan(s_, k_, t_, K_);
                    capture(b, c_);
                    const float ms = time_graph(b);
                    if (nc < CSL_BATCH_MAX_CANDIDATES) {
                        b->info.cand_slab[nc] = s_;
                        b->info.cand_ctas[nc] = c_;
                        b->info.cand_kernel[nc] = k_;
                        b->info.cand_tile[nc] = t_;
                        b->info.cand_stage[nc] = K_;
                        b->info.cand_ms[nc] = ms;
                        ++nc;
                    }
                    if (ms < best) {
                        best = ms;
                        bc = TuneChoice{s_, c_, k_, t_, K_};
                    }
                };
                // 1. field kernel and tile, at the default slab depth
                try_one(S0, 4, CSL_FIELD_BLOCK, 16, 256);
                try_one(S0, 4, CSL_FIELD_FOOTPRINT, 32, 256);
                try_one(S0, 4, CSL_FIELD_FOOTPRINT, 16, 256);
                // 2. slab depth x CTAs per SM for the best of them
                const TuneChoice k1 = bc;
                const int slabs[3] = {2, 4, 8};
                for (int si = 0; si < 3; ++si) {
                    if (slabs[si] > min_layers && slabs[si] != 2) continue;
                    const int cand_c[3] = {2, 4, 6};
                    for (int ci = 0; ci < 3; ++ci) {
                        if (k1.kernel == CSL_FIELD_FOOTPRINT && cand_c[ci] > 4) continue;
                        if (slabs[si] == S0 && cand_c[ci] == 4) continue;   // timed in step 1
                        try_one(slabs[si], cand_c[ci], k1.kernel, k1.T, 256);
                    }
                }
                // 3. the footprint kernel's staging chunk
                if (bc.kernel == CSL_FIELD_FOOTPRINT) {
                    const TuneChoice k2 = bc;
                    for (int kk : {128, 512}) try_one(k2.S, k2.ctas, k2.kernel, k2.T, kk);
                }
                b->info.n_candidates = nc;
                S = bc.S;
                ctas = bc.ctas;
                kernel = bc.kernel;
                T = bc.T;
                K = bc.K;
                plan(S, kernel, T, K);
                capture(b, ctas);
                b->info.plan_ms = plan_ms;
                b->info.tune_ms = now_ms() - t0 - plan_ms;
                std::lock_guard<std::mutex> lk(g_tune_cache_mu());
                g_tune_cache[key] = TuneChoice{S, ctas, kernel, T, K};
            } else {
                const double tp = now_ms();
                b->ctas = ctas;
                plan_jobs(b, S, kernel, T, K);
                b->info.plan_ms = now_ms() - tp;
                capture(b, ctas);
            }
            b->info.slab = b->S;
            b->info.ctas_per_sm = b->ctas;
            b->info.field_kernel = b->kernel;
            b->info.tile = b->T;
            b->info.stage_records = b->K;
            CSL_CUDA(cudaStreamSynchronize(b->st));
        } catch (...) {
            delete b;
            throw;
        }
        *out = b;
    });
}

csl_status csl_batch_run(csl_batch* b, void* stream) {
    return guard([&] {
        require_arg(b != nullptr, "batch is NULL");
        require_arg(b->exec != nullptr, "batch has no graph");
        launch_and_check(b, (cudaStream_t)stream);
    });
}

csl_status csl_batch_contours(const csl_batch* b, int32_t job, int32_t dst_on_device,
                              csl_contours** out) {
    return guard([&] {
        require_arg(out != nullptr, "out is NULL");
        *out = nullptr;
        const auto& J = job_at(b, job);
        const bool on_dev = dst_on_device != 0;
        const size_t nl = (size_t)J.d.n_layers + 1, nlo = (size_t)J.cont.n_loops + 1;
        const size_t nv = (size_t)J.cont.n_verts;
        csl_contours* c = nullptr;
        if (on_dev) {
            c = new csl_contours();
            memset(c, 0, sizeof(*c));
            c->n_layers = J.d.n_layers;
            c->on_device = 1;
            c->n_loops = J.cont.n_loops;
            c->n_verts = J.cont.n_verts;
        } else {
            c = new_host_contours(J.d.n_layers, J.cont.n_loops, J.cont.n_verts, J.want_eid);
        }
        try {
            auto alloc = [&](void** p, size_t bytes) {
                if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
                    cudaGetLastError();
                    fail(CSL_ERR_OOM, "device allocation of the contours failed");
                }
            };
            if (on_dev) {
                alloc((void**)&c->layer_loop_off, nl * 8);
                alloc((void**)&c->loop_vert_off, nlo * 8);
                alloc((void**)&c->xy, nv * 8);
                if (J.want_eid) alloc((void**)&c->edge_id, nv * 4);
            }
            const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            CSL_CUDA(cudaMemcpyAsync(c->layer_loop_off, J.cont.layer_loops.get(), nl * 8, kind,
                                     b->st));
            CSL_CUDA(cudaMemcpyAsync(c->loop_vert_off, J.cont.loop_off.get(), nlo * 8, kind,
                                     b->st));
            if (nv) {
                CSL_CUDA(cudaMemcpyAsync(c->xy, J.cont.xy.get(), nv * 8, kind, b->st));
                if (J.want_eid)
                    CSL_CUDA(cudaMemcpyAsync(c->edge_id, J.cont.eid.get(), nv * 4, kind, b->st));
            }
            CSL_CUDA(cudaStreamSynchronize(b->st));
        } catch (...) {
            csl_contours_free(c);
            throw;
        }
        *out = c;
    });
}

csl_status csl_batch_sigma(const csl_batch* b, int32_t job, float** out) {
    return guard([&] {
        require_arg(out != nullptr, "out is NULL");
        *out = job_at(b, job).sigma;
    });
}

csl_status csl_batch_get_info(const csl_batch* b, csl_batch_info* out) {
    return guard([&] {
        require_arg(b != nullptr && out != nullptr, "NULL argument");
        *out = b->info;
    });
}

void csl_batch_free(csl_batch* b) { delete b; }

}  // extern "C"
