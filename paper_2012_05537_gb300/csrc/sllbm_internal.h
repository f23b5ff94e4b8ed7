// Internal definitions shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sllbm.h"
#include "tables.h"

// The opaque context behind sllbm_ctx*.
struct sllbm_ctx {
    int cells[3];
    int N[3];
    int p;
    double L[3];
    double h[3];
    long long nn;          // nodes
    sllbm_params prm;
    double dt, U0, mu_inf, max_xi, tgv_C;
    double xi[sllbm::kQ][3];
    double w[sllbm::kQ];
    sllbm::DirTable dir[3];
    int max_shift;
    cudaStream_t stream;
    int device;
    void* buf[2];
    int cur;               // index of the buffer holding the current state
    bool own_buf;
    bool initialised;
    size_t elem;           // bytes per stored population value
    size_t pop_bytes;
    double* d_coords[3];   // node coordinates per direction (device)
    int* d_flag;           // [0] non-finite flag, [1] wait gave up (2) / abort honoured (4), [2] abort request
    cudaStream_t ctl_stream;   // side stream of sllbm_request_abort
    unsigned long long wait_ns;  // limit of the TMA-fed kernel's consumer waits
    long long steps;       // steps taken since initialisation (or the loaded checkpoint's count)
    double* d_partials;    // diagnostics partial sums (device scratch)
    double* diag_scratch;  // device address of sllbm_diag_noalloc's static array on `device`
    int partial_blocks;
    unsigned char* step_blob;  // StepTables<C,P> of the storage type, built on first step
    size_t step_blob_size;
    int num_sms;
    int step_kernel;           // 1: generic tile kernel, 2: TMA-fed persistent kernel
    int tile_shape;            // generic FP32 kernel: 0 default tile, 1 and 2 the alternatives
    int compensated;           // FP32 arithmetic: compensated moment sums (sllbm_set_compensated)
    alignas(64) unsigned char tmap[2][8][128];  // TMA descriptors (CUtensorMap) per source buffer and box shape
    const void* tmap_src[2];
    int last_err;
    long long launches;
    double tuned_ms;           // step time of the variant sllbm_autotune chose (0: not tuned)
    void* adj_buf[2];          // reverse-mode scratch (state-sized), allocated on first use
    double* d_adj_partials;    // per-block partials of the mu_inf sensitivity
    int adj_blocks;
    size_t adj_bytes;          // size of each reverse-mode scratch buffer
    bool adj_f64;              // FP32 storage with FP64 adjoint populations
    void* pipe_buf[6];         // sllbm_run_host_many: three device slots of two buffers
    cudaStream_t pipe_stream[2];  // its host-to-device and device-to-host copy streams
    cudaEvent_t pipe_ev[9];    // per slot: copied in, stepped, copied out
    // z-slab of a decomposed mesh (sllbm_create_slab): the state holds the interior cells
    // [z_begin, z_begin + cells[2]) of a mesh of z_cells_global cells along z, plus `ghost`
    // cells of halo below and above them (N[2] = (cells[2] + 2 ghost) p planes).  An ordinary
    // periodic context has slab = 0, ghost = 0.
    int slab;
    int z_begin;
    int z_cells_global;
    int ghost;
    int region;  // tiles a slab's step launches: 0 all, 1 those reading no ghost cell, 2 the others
};

namespace sllbm {

// Device allocation of the library (runtime.cu): cudaMalloc, unless sllbm_debug_fail_allocs
// armed a failure for this allocation.
cudaError_t dev_alloc_raw(void** p, size_t bytes);
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
    return dev_alloc_raw(reinterpret_cast<void**>(p), bytes);
}

// The context's two state buffers, allocated on first use unless the caller gave them (api.cu).
int ensure_buffers(sllbm_ctx* ctx);

// Step kernel for the context's parameters: 1 generic, 2 TMA-fed, 0 the requested one cannot run (api.cu).
int choose_step_kernel(const sllbm_ctx* c);

// Default limit of a bounded device-side wait.
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;

// Constant tables of the fused step, passed to the kernel by value (constant bank).
// kc[i][d][a] is the departure cell shift minus kmin[i][d] (0 or 1): the source box of a
// tile starts kmin cells away and spans span+1 extra cells.
template <typename C, int P>
struct StepTables {
    C lw[kQ][3][P][P + 1];
    signed char kc[kQ][3][P];
    signed char kmin[kQ][3];
    signed char span[kQ][3];
    C xi[kQ][3];
    C w[kQ];
};

// The velocity set (xi_i, w_i) in a compute type; the same for every context.
template <typename C>
struct Lattice {
    C xi[kQ][3];
    C w[kQ];
};

struct StepArgs {
    const void* src;
    void* dst;
    int N[3];
    int cells[3];
    int tiles[3];
    long long nn;
    double mu_over_dt;  // mu_inf / dt
    double inv_2cv;     // 1 / (2 C_v)
    double gfac;        // 2 C_v - D
    double inv_pr;      // 1 / Pr
    int pr;             // Prandtl term on
    double rho0, T0;    // reference state of 16-bit deviation storage
    int collide;        // 0: stream only
    int* flag;          // non-finite flag or nullptr
    int* flag_err;      // set (bit 2) when a bounded device-side wait gave up, (bit 4) on an honoured abort
    const int* abort_req;  // host-written abort request word (device memory) or nullptr
    unsigned long long wait_ns;  // limit of the consumers' bounded waits
    int z0;             // first interior cell along z (a slab's ghost cells; 0 on a periodic mesh)
    int tz_begin;       // first z-tile of this launch (a part of a slab's tiles; 0 otherwise)
};

// The z-tile ranges [r[k][0], r[k][1]) (k < return value) that a step launches for
// ctx->region with tiles of CZ cells.  Tile t covers the interior cells [t CZ, t CZ + tcz);
// its source boxes start at least max_shift cells below it and end with the first node of
// the cell at most max_shift cells above its last cell, so it reads no ghost cell when
// t CZ >= max_shift and t CZ + tcz + max_shift < cells.  Region 1: those tiles; region 2:
// the tiles below and above them; region 0: all tiles.
inline int slab_tile_ranges(const sllbm_ctx* c, int CZ, int r[2][2]) {
    const int ntz = (c->cells[2] + CZ - 1) / CZ;
    if (c->region == 0) {
        r[0][0] = 0;
        r[0][1] = ntz;
        return 1;
    }
    const int ms = c->max_shift;
    const int lo = (ms + CZ - 1) / CZ;
    int hi = c->cells[2] - ms - 1 >= 0 ? (c->cells[2] - ms - 1) / CZ : 0;
    if (hi > ntz) hi = ntz;
    if (hi <= lo) {  // no tile avoids the ghost cells
        if (c->region == 1) return 0;
        r[0][0] = 0;
        r[0][1] = ntz;
        return 1;
    }
    if (c->region == 1) {
        r[0][0] = lo;
        r[0][1] = hi;
        return 1;
    }
    int n = 0;
    if (lo > 0) {
        r[n][0] = 0;
        r[n][1] = lo;
        ++n;
    }
    if (hi < ntz) {
        r[n][0] = hi;
        r[n][1] = ntz;
        ++n;
    }
    return n;
}

template <typename C, int P>
void fill_step_tables(const sllbm_ctx* ctx, StepTables<C, P>* t) {
    for (int i = 0; i < kQ; ++i) {
        for (int d = 0; d < 3; ++d) {
            int kmn = 1 << 20, kmx = -(1 << 20);
            for (int a = 0; a < P; ++a) {
                int k = ctx->dir[d].shift[i][a];
                kmn = k < kmn ? k : kmn;
                kmx = k > kmx ? k : kmx;
            }
            t->kmin[i][d] = static_cast<signed char>(kmn);
            t->span[i][d] = static_cast<signed char>(kmx - kmn);
            for (int a = 0; a < P; ++a) {
                t->kc[i][d][a] = static_cast<signed char>(ctx->dir[d].shift[i][a] - kmn);
                for (int j = 0; j <= P; ++j) t->lw[i][d][a][j] = static_cast<C>(ctx->dir[d].weight[i][a][j]);
            }
            t->xi[i][d] = static_cast<C>(ctx->xi[i][d]);
        }
        t->w[i] = static_cast<C>(ctx->w[i]);
    }
}

// Step launchers, one per storage type (step_f32.cu, step_f64.cu).
int launch_step_f32(sllbm_ctx* ctx, const void* src, void* dst);
int launch_step_tma(sllbm_ctx* ctx, const void* src, void* dst);  // TMA-fed kernel, FP32 and 16-bit, p = 2..4 (step_tma.cu)
int launch_step_f64(sllbm_ctx* ctx, const void* src, void* dst);
int launch_step_f16(sllbm_ctx* ctx, const void* src, void* dst);  // both 16-bit deviation types (step_f16.cu)
// Generic FP32 kernel with one of the alternative tile shapes 1, 2 (step_f32_tiles.cu).
int launch_step_f32_shape(sllbm_ctx* ctx, const void* src, void* dst, int shape);

void fill_step_args(const sllbm_ctx* ctx, const void* src, void* dst, StepArgs* a);

// One step on ctx->stream: launch the context's step kernel from buf[cur] into buf[1-cur]
// and swap (api.cu).  No flag handling, no synchronisation.
int step_launch(sllbm_ctx* ctx);

// One mesh of a persistent batched launch: args[parity] are its step arguments from buffer
// `parity` of its ping-pong pair (parity alternates between launches); its tiles are the
// work items [tile_begin, next job's tile_begin).
struct BatchJob {
    StepArgs args[2];
    long long tile_begin;
};

// Persistent batched FP32 step of many meshes of order p (batch_kernel.cu).  Tile shapes
// (cells): 0 the generic kernel's default, 1 one size smaller, 2 one cell.
void batch_tile_cells(int p, int shape, int cells[3]);
size_t batch_tables_bytes(int p);                              // sizeof(StepTables<float, p>)
void batch_fill_tables(const sllbm_ctx* ctx, void* host_dst);  // StepTables<float, ctx->p>
int batch_group_grid(int p, int shape, int num_sms, long long items, int* grid);
int launch_batch_group(int p, int shape, const BatchJob* jobs, int njobs, const void* tabs, long long items,
                       int parity, int grid, cudaStream_t stream);

// True when the TMA-fed kernel can run this context (step_tma.cu).
bool tma_step_eligible(const sllbm_ctx* c);

// Reverse-mode scratch of a context (adjoint.cu): allocation on first use, release.
int ensure_adjoint_scratch(sllbm_ctx* ctx);
void adjoint_release(sllbm_ctx* ctx);

}  // namespace sllbm
