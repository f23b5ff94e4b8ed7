// Kernel choice, autotuner and batched (graph-captured) launch of many SLLBM contexts.
// Host code only: the kernels are the step kernels of step_f32.cu / step_f64.cu /
// step_f16.cu, launched through step_launch().
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <new>
#include <numeric>
#include <vector>

#include "sllbm_internal.h"

using namespace sllbm;

struct sllbm_batch {
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
        if (ctx->prm.storage != SLLBM_F32 || ctx->prm.pr_correction) return SLLBM_EINVAL;
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

void destroy_batch(sllbm_batch* b) {
    if (b == nullptr) return;
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
    const int v0 = current_variant(ctx);
    void* saved = nullptr;
    cudaError_t e = cudaMalloc(&saved, ctx->pop_bytes);
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
        if (c == nullptr || !c->initialised || c->prm.nonfinite_check || c->device != dev) return SLLBM_EINVAL;
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
    for (int k = 0; k < n; ++k) b->ctx[k]->launches += nsteps;
    return SLLBM_OK;
}

void sllbm_batch_destroy(sllbm_batch* b) { destroy_batch(b); }

}  // extern "C"
