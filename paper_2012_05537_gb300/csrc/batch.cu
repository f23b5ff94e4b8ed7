// Kernel choice, autotuner and batched (graph-captured) launch of many SLLBM contexts.
// Host code only: the kernels are the step kernels of step_tma.cu / step_f32.cu /
// step_f64.cu / step_f16.cu, launched through step_launch(), and the persistent batched
// kernels of batch_kernel.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <new>
#include <numeric>
#include <vector>

#include "sllbm_internal.h"
#include "trace.h"

using namespace sllbm;

// One order's share of a persistent batch: its job list and tables on the device.
struct BatchGroup {
    int p = 0, shape = 0, grid = 1, njobs = 0;
    long long items = 0;
    BatchJob* d_jobs = nullptr;
    void* d_tabs = nullptr;
    std::vector<int> members;  // indices into sllbm_batch::ctx
};

struct sllbm_batch {
    std::vector<BatchGroup> groups;  // persistent batches only
    std::vector<sllbm_ctx*> ctx;
    std::vector<int> parity;     // ctx->cur when the graph was captured
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> join;
    std::vector<cudaEvent_t> ready;  // one per context: orders the graph after its stream
    cudaEvent_t fork = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int set_variant(sllbm_ctx* ctx, int v) {
    if (v == 0) {
        if (!tma_step_eligible(ctx)) return SLLBM_EINVAL;
        ctx->step_kernel = 2;
        ctx->tile_shape = 0;
        return SLLBM_OK;
    }
    if (v == 1) {
        ctx->step_kernel = 1;
        ctx->tile_shape = 0;
        return SLLBM_OK;
    }
    if (v == 2 || v == 3) {
        if (ctx->prm.storage != SLLBM_F32 || ctx->prm.pr_correction || ctx->compensated) return SLLBM_EINVAL;
        ctx->step_kernel = 1;
        ctx->tile_shape = v - 1;
        return SLLBM_OK;
    }
    return SLLBM_EINVAL;
}

int current_variant(const sllbm_ctx* ctx) { return ctx->step_kernel == 2 ? 0 : 1 + ctx->tile_shape; }

int cuda_fail(sllbm_ctx* ctx, cudaError_t e) {
    if (ctx) ctx->last_err = static_cast<int>(e);
    return SLLBM_ECUDA;
}

void free_group(BatchGroup& g) {
    cudaFree(g.d_jobs);
    cudaFree(g.d_tabs);
    g.d_jobs = nullptr;
    g.d_tabs = nullptr;
}

// Builds the job list and tables of group g for its tile shape (synchronous copies).
int build_group(BatchGroup& g, const std::vector<sllbm_ctx*>& ctx, int num_sms) {
    free_group(g);
    int tc[3];
    batch_tile_cells(g.p, g.shape, tc);
    std::vector<BatchJob> jobs(g.members.size());
    const size_t tb = batch_tables_bytes(g.p);
    std::vector<unsigned char> tabs(tb * g.members.size());
    long long items = 0;
    for (size_t k = 0; k < g.members.size(); ++k) {
        const sllbm_ctx* c = ctx[g.members[k]];
        for (int par = 0; par < 2; ++par) {
            const int from = par == 0 ? c->cur : 1 - c->cur;
            fill_step_args(c, c->buf[from], c->buf[1 - from], &jobs[k].args[par]);
            jobs[k].args[par].flag = nullptr;
            for (int d = 0; d < 3; ++d) jobs[k].args[par].tiles[d] = (c->cells[d] + tc[d] - 1) / tc[d];
        }
        jobs[k].tile_begin = items;
        items += static_cast<long long>(jobs[k].args[0].tiles[0]) * jobs[k].args[0].tiles[1] * jobs[k].args[0].tiles[2];
        batch_fill_tables(c, tabs.data() + tb * k);
    }
    g.njobs = static_cast<int>(jobs.size());
    g.items = items;
    cudaError_t e = dev_alloc(&g.d_jobs, sizeof(BatchJob) * jobs.size());
    if (e == cudaSuccess) e = dev_alloc(&g.d_tabs, tabs.size());
    if (e == cudaSuccess) e = cudaMemcpy(g.d_jobs, jobs.data(), sizeof(BatchJob) * jobs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_tabs, tabs.data(), tabs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_group(g);
        return e == cudaErrorMemoryAllocation ? SLLBM_ENOMEM : SLLBM_ECUDA;
    }
    return batch_group_grid(g.p, g.shape, num_sms, items, &g.grid);
}

void destroy_batch(sllbm_batch* b) {
    if (b == nullptr) return;
    for (BatchGroup& g : b->groups) free_group(g);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ready) cudaEventDestroy(e);
    for (cudaStream_t s : b->workers) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

}  // namespace

extern "C" {

int sllbm_set_step_variant(sllbm_ctx* ctx, int variant) {
    if (ctx == nullptr) return SLLBM_EINVAL;
    return set_variant(ctx, variant);
}

int sllbm_autotune(sllbm_ctx* ctx, int steps, int* variant, double* ms_per_step) {
    if (ctx == nullptr || steps < 1) return SLLBM_EINVAL;
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    const int cur0 = ctx->cur;
    const long long steps0 = ctx->steps;
    const int v0 = current_variant(ctx);
    void* saved = nullptr;
    cudaError_t e = dev_alloc(&saved, ctx->pop_bytes);
    if (e != cudaSuccess) {
        ctx->last_err = static_cast<int>(e);
        return SLLBM_ENOMEM;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int rc = SLLBM_OK;
    int best = -1;
    float best_ms = 0.0f;
    e = cudaMemcpyAsync(saved, ctx->buf[cur0], ctx->pop_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e);
    for (int v = 0; v < 4 && rc == SLLBM_OK; ++v) {
        if (set_variant(ctx, v) != SLLBM_OK) continue;
        ctx->cur = cur0;
        e = cudaMemcpyAsync(ctx->buf[cur0], saved, ctx->pop_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(ctx, e);
            break;
        }
        rc = step_launch(ctx);  // warm-up (tables, descriptors, function attributes)
        if (rc == SLLBM_OK) e = cudaEventRecord(ev[0], ctx->stream);
        for (int s = 0; s < steps && rc == SLLBM_OK && e == cudaSuccess; ++s) rc = step_launch(ctx);
        if (rc != SLLBM_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) {
            rc = cuda_fail(ctx, e);
            break;
        }
        ms /= static_cast<float>(steps);
        if (best < 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    // the state as it was, in the buffer it was in
    ctx->cur = cur0;
    ctx->steps = steps0;
    cudaError_t e2 = cudaMemcpyAsync(ctx->buf[cur0], saved, ctx->pop_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(ctx->stream);
    if (e2 != cudaSuccess && rc == SLLBM_OK) rc = cuda_fail(ctx, e2);
    cudaFree(saved);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (rc != SLLBM_OK || best < 0) {
        set_variant(ctx, v0);
        return rc != SLLBM_OK ? rc : SLLBM_EINVAL;
    }
    set_variant(ctx, best);
    ctx->tuned_ms = best_ms;
    if (variant) *variant = best;
    if (ms_per_step) *ms_per_step = best_ms;
    return SLLBM_OK;
}

int sllbm_batch_plan(const double* cost, int n, int streams, int* assign) {
    if (cost == nullptr || assign == nullptr || n < 1 || streams < 1) return SLLBM_EINVAL;
    for (int k = 0; k < n; ++k)
        if (!(cost[k] >= 0.0)) return SLLBM_EINVAL;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(streams, 0.0);
    for (int k : order) {
        int w = 0;
        for (int s = 1; s < streams; ++s)
            if (load[s] < load[w]) w = s;
        assign[k] = w;
        load[w] += cost[k];
    }
    return SLLBM_OK;
}

int sllbm_batch_create(sllbm_ctx* const* ctxs, int n, int streams, void* cuda_stream, sllbm_batch** out) {
    if (out == nullptr) return SLLBM_EINVAL;
    *out = nullptr;
    // the legacy default stream cannot be captured into a graph
    if (ctxs == nullptr || n < 1 || streams < 1 || cuda_stream == nullptr) return SLLBM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLLBM_ECUDA;
    for (int k = 0; k < n; ++k) {
        const sllbm_ctx* c = ctxs[k];
        // (a slab needs its halo exchanged between steps: not inside a batch)
        if (c == nullptr || !c->initialised || c->prm.nonfinite_check || c->device != dev || c->slab)
            return SLLBM_EINVAL;
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c) return SLLBM_EINVAL;
    }
    if (streams > n) streams = n;
    sllbm_batch* b = new (std::nothrow) sllbm_batch;
    if (b == nullptr) return SLLBM_ENOMEM;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    // per-step cost estimate: autotuned times when every context has one, else node counts
    bool all_tuned = true;
    for (int k = 0; k < n; ++k) all_tuned = all_tuned && ctxs[k]->tuned_ms > 0.0;
    std::vector<double> cost(n);
    for (int k = 0; k < n; ++k) cost[k] = all_tuned ? ctxs[k]->tuned_ms : static_cast<double>(ctxs[k]->nn);
    std::vector<int> assign(n);
    sllbm_batch_plan(cost.data(), n, streams, assign.data());

    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    for (int s = 0; s < streams && e == cudaSuccess; ++s) {
        cudaStream_t w = nullptr;
        cudaEvent_t j = nullptr;
        e = cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->workers.push_back(w);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(j);
    }
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        cudaEvent_t r = nullptr;
        e = cudaEventCreateWithFlags(&r, cudaEventDisableTiming);
        if (e == cudaSuccess) b->ready.push_back(r);
    }
    if (e != cudaSuccess) {
        destroy_batch(b);
        return SLLBM_ECUDA;
    }

    // Two steps per context (the ping-pong parity returns to where it was), captured with the
    // contexts temporarily on their worker streams.  Relaxed mode: the launchers may set
    // function attributes and build host-side descriptors while capturing.
    std::vector<cudaStream_t> own(n);
    std::vector<long long> launches(n);
    for (int k = 0; k < n; ++k) {
        own[k] = ctxs[k]->stream;
        launches[k] = ctxs[k]->launches;
        b->parity.push_back(ctxs[k]->cur);
    }
    int rc = SLLBM_OK;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    for (int s = 0; s < streams && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->workers[s], b->fork, 0);
    for (int k = 0; k < n && e == cudaSuccess && rc == SLLBM_OK; ++k) {
        sllbm_ctx* c = ctxs[k];
        c->stream = b->workers[assign[k]];
        rc = step_launch(c);
        if (rc == SLLBM_OK) rc = step_launch(c);
        c->stream = own[k];
    }
    for (int s = 0; s < streams && e == cudaSuccess && rc == SLLBM_OK; ++s) {
        e = cudaEventRecord(b->join[s], b->workers[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[s], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e_end = cudaStreamEndCapture(b->stream, &g);
    for (int k = 0; k < n; ++k) {
        ctxs[k]->cur = b->parity[k];
        ctxs[k]->launches = launches[k];
    }
    if (rc == SLLBM_OK && e == cudaSuccess && e_end == cudaSuccess) {
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    } else {
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = e_end;
    }
    if (rc != SLLBM_OK || e != cudaSuccess) {
        cudaGetLastError();  // clear a capture error so the contexts stay usable
        destroy_batch(b);
        return rc != SLLBM_OK ? rc : SLLBM_ECUDA;
    }
    *out = b;
    return SLLBM_OK;
}

int sllbm_batch_step(sllbm_batch* b, int nsteps) {
    NvtxRange range("sllbm_batch_step");
    if (b == nullptr || nsteps < 0 || (nsteps & 1)) return SLLBM_EINVAL;
    const int n = static_cast<int>(b->ctx.size());
    for (int k = 0; k < n; ++k)
        if (b->ctx[k]->cur != b->parity[k]) return SLLBM_EINVAL;
    if (nsteps == 0) return SLLBM_OK;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        if (b->ctx[k]->stream == b->stream) continue;
        e = cudaEventRecord(b->ready[k], b->ctx[k]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ready[k], 0);
    }
    for (int r = 0; r < nsteps / 2 && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        if (b->ctx[k]->stream != b->stream) e = cudaStreamWaitEvent(b->ctx[k]->stream, b->done, 0);
    }
    if (e != cudaSuccess) return cuda_fail(b->ctx[0], e);
    if (b->groups.empty())
        for (int k = 0; k < n; ++k) b->ctx[k]->launches += nsteps;
    return SLLBM_OK;
}

// Captures two steps of every group (each on its worker stream, parity 0 then 1) into
// b->graph and instantiates b->exec, replacing a previous graph.
static int capture_persistent(sllbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    int rc = SLLBM_OK;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    for (size_t s = 0; s < b->groups.size() && e == cudaSuccess && rc == SLLBM_OK; ++s) {
        const BatchGroup& g = b->groups[s];
        e = cudaStreamWaitEvent(b->workers[s], b->fork, 0);
        for (int par = 0; par < 2 && e == cudaSuccess && rc == SLLBM_OK; ++par)
            rc = launch_batch_group(g.p, g.shape, g.d_jobs, g.njobs, g.d_tabs, g.items, par, g.grid, b->workers[s]);
        if (e == cudaSuccess && rc == SLLBM_OK) e = cudaEventRecord(b->join[s], b->workers[s]);
        if (e == cudaSuccess && rc == SLLBM_OK) e = cudaStreamWaitEvent(b->stream, b->join[s], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(b->stream, &graph);
    if (rc == SLLBM_OK && e == cudaSuccess && e_end == cudaSuccess) {
        b->graph = graph;
        if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = SLLBM_ECUDA;
    } else {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (rc == SLLBM_OK) rc = SLLBM_ECUDA;
    }
    return rc;
}

int sllbm_batch_create_persistent(sllbm_ctx* const* ctxs, int n, void* cuda_stream, int tune_steps,
                                  sllbm_batch** out) {
    if (out == nullptr) return SLLBM_EINVAL;
    *out = nullptr;
    if (ctxs == nullptr || n < 1 || cuda_stream == nullptr || tune_steps < 0) return SLLBM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLLBM_ECUDA;
    for (int k = 0; k < n; ++k) {
        const sllbm_ctx* c = ctxs[k];
        // (a slab needs its halo exchanged between steps: not inside a batch)
        if (c == nullptr || !c->initialised || c->prm.nonfinite_check || c->device != dev || c->slab)
            return SLLBM_EINVAL;
        if (c->prm.storage != SLLBM_F32 || c->prm.pr_correction || !c->prm.collide || c->compensated)
            return SLLBM_EINVAL;
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c) return SLLBM_EINVAL;
    }
    sllbm_batch* b = new (std::nothrow) sllbm_batch;
    if (b == nullptr) return SLLBM_ENOMEM;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int k = 0; k < n; ++k) b->parity.push_back(ctxs[k]->cur);
    for (int p = 2; p <= 4; ++p) {
        BatchGroup g;
        g.p = p;
        for (int k = 0; k < n; ++k)
            if (ctxs[k]->p == p) g.members.push_back(k);
        if (!g.members.empty()) b->groups.push_back(g);
    }
    const int num_sms = ctxs[0]->num_sms;
    int rc = SLLBM_OK;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    for (size_t s = 0; s < b->groups.size() && e == cudaSuccess; ++s) {
        cudaStream_t w = nullptr;
        cudaEvent_t j = nullptr;
        e = cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->workers.push_back(w);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(j);
    }
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        cudaEvent_t r = nullptr;
        e = cudaEventCreateWithFlags(&r, cudaEventDisableTiming);
        if (e == cudaSuccess) b->ready.push_back(r);
    }
    if (e != cudaSuccess) rc = SLLBM_ECUDA;

    // Autotuner: the groups run concurrently in the graph (one worker stream each), so they
    // are timed together, `tune_steps` (rounded up to even) steps of all groups from the
    // current states; a coordinate descent over the groups keeps another tile shape for a
    // group only if all groups then run at least 2 % faster.  The states are restored.
    for (size_t s = 0; s < b->groups.size() && rc == SLLBM_OK; ++s) {
        b->groups[s].shape = 0;
        rc = build_group(b->groups[s], b->ctx, num_sms);
    }
    if (rc == SLLBM_OK && tune_steps > 0) {
        const int steps = tune_steps + (tune_steps & 1);
        std::vector<void*> saved(n, nullptr);
        for (int k = 0; k < n && rc == SLLBM_OK; ++k) {
            e = dev_alloc(&saved[k], ctxs[k]->pop_bytes);
            if (e == cudaSuccess)
                e = cudaMemcpy(saved[k], ctxs[k]->buf[ctxs[k]->cur], ctxs[k]->pop_bytes, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? SLLBM_ENOMEM : SLLBM_ECUDA;
        }
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (rc == SLLBM_OK && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess))
            rc = SLLBM_ECUDA;
        // the graph of the current shapes, replayed: 2 steps of warm-up, then `steps` timed
        auto time_graph = [&](float* ms) -> int {
            int r = capture_persistent(b);
            if (r != SLLBM_OK) return r;
            if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return SLLBM_ECUDA;
            if (cudaEventRecord(ev[0], b->stream) != cudaSuccess) return SLLBM_ECUDA;
            for (int s2 = 0; s2 < steps / 2; ++s2)
                if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return SLLBM_ECUDA;
            if (cudaEventRecord(ev[1], b->stream) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                cudaEventElapsedTime(ms, ev[0], ev[1]) != cudaSuccess)
                return SLLBM_ECUDA;
            return SLLBM_OK;
        };
        float best_ms = 0.0f;
        if (rc == SLLBM_OK) rc = time_graph(&best_ms);
        for (size_t g = 0; g < b->groups.size() && rc == SLLBM_OK; ++g) {
            BatchGroup& gr = b->groups[g];
            int best = gr.shape;
            for (int sh = 1; sh < 3 && rc == SLLBM_OK; ++sh) {
                gr.shape = sh;
                rc = build_group(gr, b->ctx, num_sms);
                float ms = 0.0f;
                if (rc == SLLBM_OK) rc = time_graph(&ms);
                if (rc == SLLBM_OK && ms < 0.98f * best_ms) {
                    best = sh;
                    best_ms = ms;
                }
            }
            if (rc != SLLBM_OK) break;
            gr.shape = best;
            rc = build_group(gr, b->ctx, num_sms);
        }
        for (int k = 0; k < n; ++k) {
            if (saved[k] != nullptr && rc == SLLBM_OK)
                if (cudaMemcpy(ctxs[k]->buf[ctxs[k]->cur], saved[k], ctxs[k]->pop_bytes, cudaMemcpyDeviceToDevice) !=
                    cudaSuccess)
                    rc = SLLBM_ECUDA;
            cudaFree(saved[k]);
        }
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
    }

    // the graph: per order, on its own worker stream, two launches (parity 0 then 1)
    if (rc == SLLBM_OK) rc = capture_persistent(b);
    if (rc != SLLBM_OK) {
        cudaGetLastError();
        destroy_batch(b);
        return rc;
    }
    *out = b;
    return SLLBM_OK;
}

int sllbm_batch_shapes(const sllbm_batch* b, int* shape_p2, int* shape_p3, int* shape_p4) {
    if (b == nullptr) return SLLBM_EINVAL;
    int* dst[3] = {shape_p2, shape_p3, shape_p4};
    for (int k = 0; k < 3; ++k)
        if (dst[k]) *dst[k] = -1;
    for (const BatchGroup& g : b->groups)
        if (dst[g.p - 2]) *dst[g.p - 2] = g.shape;
    return SLLBM_OK;
}

void sllbm_batch_destroy(sllbm_batch* b) { destroy_batch(b); }

}  // extern "C"
