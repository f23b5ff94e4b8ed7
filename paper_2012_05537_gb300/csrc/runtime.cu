// Run control around the step (the paper describes none of this): device allocation with a
// host-side failure injector, the consumer wait limit and the abort request of the
// persistent TMA-fed kernel, and checkpoints of a context's state with a self-describing
// header.  Declared in include/sllbm.h; the checkpoint layout is sllbm_checkpoint_t there.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "sllbm_internal.h"

namespace sllbm {

namespace {
// Allocations left before the injected failure; -1: no failure armed.
std::atomic<long long> g_alloc_fail_after{-1};
}  // namespace

cudaError_t dev_alloc_raw(void** p, size_t bytes) {
    long long v = g_alloc_fail_after.load();
    while (v >= 0) {
        if (g_alloc_fail_after.compare_exchange_weak(v, v - 1)) {
            if (v == 0) {  // this is the allocation that fails; the injector disarms itself
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

}  // namespace sllbm

using namespace sllbm;

namespace {

constexpr char kMagic[8] = {'S', 'L', 'L', 'B', 'M', 'C', 'K', '1'};
constexpr uint32_t kVersion = 1;

struct CkptHeader {  // 128 bytes, host byte order
    char magic[8];
    uint32_t version;
    int32_t storage;
    int32_t p;
    int32_t velset;
    int32_t cells[3];
    int32_t pr_correction;
    double L[3];
    double dt;
    double mu_inf;
    double rho0;
    double T0;
    int64_t steps;
    uint64_t payload_bytes;
    unsigned char reserved[16];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header layout");

// Reads and checks the header of a checkpoint file; leaves the file positioned at the payload.
int read_header(FILE* f, CkptHeader* h) {
    if (std::fread(h, sizeof(*h), 1, f) != 1) return SLLBM_EINVAL;
    if (std::memcmp(h->magic, kMagic, sizeof(kMagic)) != 0 || h->version != kVersion) return SLLBM_EINVAL;
    if (h->p < 2 || h->p > 4 || h->storage < SLLBM_F64 || h->storage > SLLBM_BF16DEV || h->velset != SLLBM_D3Q45)
        return SLLBM_EINVAL;
    unsigned long long nodes = 1;
    for (int d = 0; d < 3; ++d) {
        if (h->cells[d] < 1) return SLLBM_EINVAL;
        nodes *= static_cast<unsigned long long>(h->cells[d]) * static_cast<unsigned long long>(h->p);
    }
    const unsigned long long elem = h->storage == SLLBM_F64 ? 8 : h->storage == SLLBM_F32 ? 4 : 2;
    if (h->payload_bytes != 2ull * kQ * nodes * elem) return SLLBM_EINVAL;
    return SLLBM_OK;
}

}  // namespace

extern "C" {

int sllbm_debug_fail_allocs(int after) {
    if (after < -1) return SLLBM_EINVAL;
    g_alloc_fail_after.store(after);
    return SLLBM_OK;
}

int sllbm_set_wait_limit(sllbm_ctx* ctx, double seconds) {
    if (ctx == nullptr || !(seconds >= 0.0) || seconds > 60.0) return SLLBM_EINVAL;
    ctx->wait_ns = static_cast<unsigned long long>(seconds * 1e9);
    return SLLBM_OK;
}

int sllbm_request_abort(sllbm_ctx* ctx, int on) {
    if (ctx == nullptr || ctx->d_flag == nullptr) return SLLBM_EINVAL;
    // written on the context's side stream, so that the word can change while steps queued on
    // the context's stream are still running; the call returns once the word is written
    const int v = on ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync(ctx->d_flag + 2, &v, sizeof(int), cudaMemcpyHostToDevice, ctx->ctl_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->ctl_stream);
    if (e != cudaSuccess) {
        ctx->last_err = static_cast<int>(e);
        return SLLBM_ECUDA;
    }
    return SLLBM_OK;
}

int64_t sllbm_step_count(const sllbm_ctx* ctx) { return ctx ? ctx->steps : 0; }

int sllbm_set_compensated(sllbm_ctx* ctx, int on) {
    if (ctx == nullptr) return SLLBM_EINVAL;
    // (the TMA-fed kernel has no instance with both compensated sums and the Prandtl term)
    if (on && ctx->prm.kernel == 2 && ctx->prm.pr_correction) return SLLBM_EINVAL;
    ctx->compensated = on ? 1 : 0;
    if (ctx->compensated) ctx->tile_shape = 0;  // the generic kernel's alternative tiles sum plainly
    ctx->step_kernel = choose_step_kernel(ctx);
    return SLLBM_OK;
}

int sllbm_save(sllbm_ctx* ctx, const char* path) {
    if (ctx == nullptr || path == nullptr || ctx->slab) return SLLBM_EINVAL;
    if (!ctx->initialised || ctx->buf[ctx->cur] == nullptr) return SLLBM_ENOTREADY;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.storage = ctx->prm.storage;
    h.p = ctx->p;
    h.velset = SLLBM_D3Q45;
    for (int d = 0; d < 3; ++d) {
        h.cells[d] = ctx->cells[d];
        h.L[d] = ctx->L[d];
    }
    h.pr_correction = ctx->prm.pr_correction;
    h.dt = ctx->dt;
    h.mu_inf = ctx->mu_inf;
    h.rho0 = ctx->prm.rho0;
    h.T0 = ctx->prm.T0;
    h.steps = ctx->steps;
    h.payload_bytes = ctx->pop_bytes;
    void* host = std::malloc(ctx->pop_bytes);
    if (host == nullptr) return SLLBM_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(host, ctx->buf[ctx->cur], ctx->pop_bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        std::free(host);
        ctx->last_err = static_cast<int>(e);
        return SLLBM_ECUDA;
    }
    FILE* f = std::fopen(path, "wb");
    int rc = SLLBM_OK;
    if (f == nullptr) {
        rc = SLLBM_EIO;
    } else {
        if (std::fwrite(&h, sizeof(h), 1, f) != 1 || std::fwrite(host, 1, ctx->pop_bytes, f) != ctx->pop_bytes)
            rc = SLLBM_EIO;
        if (std::fclose(f) != 0) rc = SLLBM_EIO;
    }
    std::free(host);
    return rc;
}

int sllbm_load(sllbm_ctx* ctx, const char* path) {
    if (ctx == nullptr || path == nullptr || ctx->slab) return SLLBM_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (f == nullptr) return SLLBM_EIO;
    CkptHeader h;
    int rc = read_header(f, &h);
    // the state only means something on the same mesh, order, storage, reference state and
    // time step (the streaming tables depend on dt)
    if (rc == SLLBM_OK) {
        bool same = h.storage == ctx->prm.storage && h.p == ctx->p && h.dt == ctx->dt &&
                    h.rho0 == ctx->prm.rho0 && h.T0 == ctx->prm.T0 && h.payload_bytes == ctx->pop_bytes;
        for (int d = 0; d < 3; ++d) same = same && h.cells[d] == ctx->cells[d] && h.L[d] == ctx->L[d];
        if (!same) rc = SLLBM_EINVAL;
    }
    void* host = nullptr;
    if (rc == SLLBM_OK) {
        host = std::malloc(ctx->pop_bytes);
        if (host == nullptr) rc = SLLBM_ENOMEM;
    }
    if (rc == SLLBM_OK && std::fread(host, 1, ctx->pop_bytes, f) != ctx->pop_bytes) rc = SLLBM_EINVAL;  // truncated
    std::fclose(f);
    if (rc == SLLBM_OK) rc = ensure_buffers(ctx);
    if (rc == SLLBM_OK) {
        cudaError_t e = cudaMemcpyAsync(ctx->buf[ctx->cur], host, ctx->pop_bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            ctx->last_err = static_cast<int>(e);
            rc = SLLBM_ECUDA;
        }
    }
    std::free(host);
    if (rc != SLLBM_OK) return rc;
    ctx->mu_inf = h.mu_inf;
    ctx->steps = h.steps;
    ctx->initialised = true;
    return SLLBM_OK;
}

int sllbm_checkpoint_info(const char* path, sllbm_checkpoint_t* out) {
    if (path == nullptr || out == nullptr) return SLLBM_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (f == nullptr) return SLLBM_EIO;
    CkptHeader h;
    int rc = read_header(f, &h);
    if (rc == SLLBM_OK) {
        // the payload must be all there
        if (std::fseek(f, 0, SEEK_END) != 0) rc = SLLBM_EIO;
        const long end = rc == SLLBM_OK ? std::ftell(f) : -1;
        if (rc == SLLBM_OK && (end < 0 || static_cast<unsigned long long>(end) != sizeof(h) + h.payload_bytes))
            rc = SLLBM_EINVAL;
    }
    std::fclose(f);
    if (rc != SLLBM_OK) return rc;
    out->storage = h.storage;
    out->p = h.p;
    out->velset = h.velset;
    for (int d = 0; d < 3; ++d) {
        out->cells[d] = h.cells[d];
        out->L[d] = h.L[d];
    }
    out->pr_correction = h.pr_correction;
    out->dt = h.dt;
    out->mu_inf = h.mu_inf;
    out->rho0 = h.rho0;
    out->T0 = h.T0;
    out->steps = h.steps;
    out->payload_bytes = h.payload_bytes;
    return SLLBM_OK;
}

}  // extern "C"
