// C ABI of the SLLBM step library (declared in include/sllbm.h) and its auxiliary
// kernels: equilibrium initialisation, population conversion, moments, diagnostics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "collide.cuh"
#include "sllbm_internal.h"
#include "trace.h"
#include "storage.cuh"
#include "tables.h"

using namespace sllbm;

namespace {

constexpr double kPi = 3.14159265358979323846;

struct VelConst {
    double xi[kQ][3];
    double w[kQ];
};

VelConst vel_const(const sllbm_ctx* ctx) {
    VelConst v;
    std::memcpy(v.xi, ctx->xi, sizeof(v.xi));
    std::memcpy(v.w, ctx->w, sizeof(v.w));
    return v;
}

int fail(sllbm_ctx* ctx, cudaError_t e) {
    if (ctx) ctx->last_err = static_cast<int>(e);
    return SLLBM_ECUDA;
}

#define CK(ctx, call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return fail((ctx), e_);       \
    } while (0)

// Calls f with a value of the storage type of the context (double, float, __half, bfloat16).
template <typename F>
void with_storage(const sllbm_ctx* ctx, F&& f) {
    switch (ctx->prm.storage) {
    case SLLBM_F64: f(double{}); break;
    case SLLBM_F32: f(float{}); break;
    case SLLBM_F16DEV: f(__half{}); break;
    default: f(__nv_bfloat16{}); break;
    }
}

// Deviation references of 16-bit storage: rho0 for f, (2 C_v - D) T0 rho0 for g.
PopRef pop_ref(const sllbm_ctx* ctx) {
    const double gfac = 2.0 / (ctx->prm.gamma - 1.0) - 3.0;
    return PopRef{ctx->prm.rho0, gfac * ctx->prm.T0 * ctx->prm.rho0};
}

unsigned grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 1048576) g = 1048576;
    if (g < 1) g = 1;
    return static_cast<unsigned>(g);
}

// ---------------------------------------------------------------- initialisation
// f_i = f_i^eq(rho, u, T), g_i = (2C_v - D) T f_i^eq, in FP64 (Eq. discreteEquilibrium).
// mode 0: Taylor-Green fields of Sec. III.C at the node coordinates; mode 1: given fields.
template <typename S>
__global__ void init_eq_kernel(S* __restrict__ pop, long long nn, int Nx, int Ny,
                               const double* __restrict__ cx, const double* __restrict__ cy,
                               const double* __restrict__ cz, int mode, double U0, double rho0,
                               double T0, double C, const double* __restrict__ rho_f,
                               const double* __restrict__ u_f, const double* __restrict__ T_f,
                               double gfac, PopRef ref, const __grid_constant__ VelConst vc) {
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x) {
        double rho, ux, uy, uz, T;
        if (mode == 0) {
            const int ix = static_cast<int>(n % Nx);
            const int iy = static_cast<int>((n / Nx) % Ny);
            const int iz = static_cast<int>(n / (static_cast<long long>(Nx) * Ny));
            const double x = cx[ix], y = cy[iy], z = cz[iz];
            ux = U0 * sin(x) * cos(y) * cos(z);
            uy = -U0 * cos(x) * sin(y) * cos(z);
            uz = 0.0;
            rho = rho0 * (1.0 + C / 16.0 * (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0));
            T = T0;
        } else {
            rho = rho_f[n];
            ux = u_f[n];
            uy = u_f[nn + n];
            uz = u_f[2 * nn + n];
            T = T_f[n];
        }
        const EqCoef<double> ec = eq_coefficients(ux * ux + uy * uy + uz * uz, T - 1.0);
#pragma unroll 5
        for (int i = 0; i < kQ; ++i) {
            const double s = vc.xi[i][0] * ux + vc.xi[i][1] * uy + vc.xi[i][2] * uz;
            const double feq = vc.w[i] * rho * eq_poly(ec, shell_of(i), s);
            pop[2 * (i * nn + n)] = PopCodec<S>::encode(feq, vc.w[i], ref.f);
            pop[2 * (i * nn + n) + 1] = PopCodec<S>::encode(gfac * T * feq, vc.w[i], ref.g);
        }
    }
}

// FP64 populations in the interface order [h][i][node] <-> the storage order
// [i][node][h] (f_i and g_i of a node side by side), rounding to the storage type.
template <typename S>
__global__ void pack_kernel(const double* __restrict__ in, S* __restrict__ out, long long nn, PopRef ref,
                            const __grid_constant__ VelConst vc) {
    const long long count = 2LL * kQ * nn;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < count;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long h = k & 1, r = k >> 1;  // r = i*nn + node
        const int i = static_cast<int>(r / nn);
        out[k] = PopCodec<S>::encode(in[h * kQ * nn + r], vc.w[i], h ? ref.g : ref.f);
    }
}

template <typename S>
__global__ void unpack_kernel(const S* __restrict__ in, double* __restrict__ out, long long nn, PopRef ref,
                              const __grid_constant__ VelConst vc) {
    const long long count = 2LL * kQ * nn;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < count;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long h = k & 1, r = k >> 1;
        const int i = static_cast<int>(r / nn);
        out[h * kQ * nn + r] = PopCodec<S>::decode(in[k], vc.w[i], h ? ref.g : ref.f);
    }
}

// ---------------------------------------------------------------- moments
template <typename S>
__global__ void moments_kernel(const S* __restrict__ pop, long long nn, double inv_2cv,
                               double* __restrict__ rho_o, double* __restrict__ u_o,
                               double* __restrict__ T_o, PopRef ref, const __grid_constant__ VelConst vc) {
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x) {
        double rho = 0, mx = 0, my = 0, mz = 0, e2 = 0;
#pragma unroll 5
        for (int i = 0; i < kQ; ++i) {
            const double f = PopCodec<S>::decode(pop[2 * (i * nn + n)], vc.w[i], ref.f);
            rho += f;
            mx += f * vc.xi[i][0];
            my += f * vc.xi[i][1];
            mz += f * vc.xi[i][2];
            e2 += f * shell_xi2(shell_of(i)) + PopCodec<S>::decode(pop[2 * (i * nn + n) + 1], vc.w[i], ref.g);
        }
        const double ux = mx / rho, uy = my / rho, uz = mz / rho;
        rho_o[n] = rho;
        u_o[n] = ux;
        u_o[nn + n] = uy;
        u_o[2 * nn + n] = uz;
        T_o[n] = (e2 / rho - (ux * ux + uy * uy + uz * uz)) * inv_2cv;
    }
}

// ---------------------------------------------------------------- diagnostics
struct DiagConst {
    double xi[kQ][3];
    double w[kQ];
    PopRef ref;
    double W[kMaxP + 1];
    double D[kMaxP + 1][kMaxP + 1];
};

// Per cell: rho, u, T at its (p+1)^3 support points, gradients from the cell-local
// Lagrange polynomials, Clenshaw-Curtis quadrature of rho|u|^2/2, mu~|curl u|^2 and
// mu~(div u)^2 (Sec. III.C).  Grid-stride over cells; one FP64 partial triple per block.
// Along z the support points wrap around within Nz planes that start zoff planes into the
// buffer (the whole buffer of a periodic context; the interior of a slab spanning the whole
// mesh, so that its ghost planes are not read).
template <typename S, int P>
__global__ void __launch_bounds__(128) diag_kernel(const S* __restrict__ pop, long long nn, int Nx, int Ny,
                                                   int Nz, int zoff, int ncx, int ncy, long long ncell,
                                                   double inv_2cv,
                                                   double hx, double hy, double hz,
                                                   const __grid_constant__ DiagConst dc,
                                                   double* __restrict__ partials) {
    constexpr int P1 = P + 1;
    constexpr int NPC = P1 * P1 * P1;
    __shared__ double su[3][NPC];
    __shared__ double red[3][4];
    double acc0 = 0, acc1 = 0, acc2 = 0;
    const int t = threadIdx.x;
    const int ia = t % P1, ib = (t / P1) % P1, ic = t / (P1 * P1);
    for (long long cell = blockIdx.x; cell < ncell; cell += gridDim.x) {
        const int cx = static_cast<int>(cell % ncx);
        const int cy = static_cast<int>((cell / ncx) % ncy);
        const int cz = static_cast<int>(cell / (static_cast<long long>(ncx) * ncy));
        double rho = 0, T = 0, ux = 0, uy = 0, uz = 0;
        if (t < NPC) {
            const int nx = (cx * P + ia) % Nx, ny = (cy * P + ib) % Ny, nz = zoff + (cz * P + ic) % Nz;
            const long long n = (static_cast<long long>(nz) * Ny + ny) * Nx + nx;
            double mx = 0, my = 0, mz = 0, e2 = 0;
            for (int i = 0; i < kQ; ++i) {
                const double f = PopCodec<S>::decode(pop[2 * (i * nn + n)], dc.w[i], dc.ref.f);
                rho += f;
                mx += f * dc.xi[i][0];
                my += f * dc.xi[i][1];
                mz += f * dc.xi[i][2];
                e2 += f * shell_xi2(shell_of(i)) + PopCodec<S>::decode(pop[2 * (i * nn + n) + 1], dc.w[i], dc.ref.g);
            }
            ux = mx / rho;
            uy = my / rho;
            uz = mz / rho;
            T = (e2 / rho - (ux * ux + uy * uy + uz * uz)) * inv_2cv;
            su[0][t] = ux;
            su[1][t] = uy;
            su[2][t] = uz;
        }
        __syncthreads();
        if (t < NPC) {
            double g[3][3];  // g[comp][dir]
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double sx = 0, sy = 0, sz = 0;
#pragma unroll
                for (int j = 0; j < P1; ++j) {
                    sx += dc.D[ia][j] * su[c][(ic * P1 + ib) * P1 + j];
                    sy += dc.D[ib][j] * su[c][(ic * P1 + j) * P1 + ia];
                    sz += dc.D[ic][j] * su[c][(j * P1 + ib) * P1 + ia];
                }
                g[c][0] = sx * 2.0 / hx;
                g[c][1] = sy * 2.0 / hy;
                g[c][2] = sz * 2.0 / hz;
            }
            const double wq = dc.W[ia] * dc.W[ib] * dc.W[ic] * hx * hy * hz * 0.125;
            const double wx = g[2][1] - g[1][2], wy = g[0][2] - g[2][0], wz = g[1][0] - g[0][1];
            const double dv = g[0][0] + g[1][1] + g[2][2];
            const double mut = sutherland(T);
            acc0 += wq * 0.5 * rho * (ux * ux + uy * uy + uz * uz);
            acc1 += wq * mut * (wx * wx + wy * wy + wz * wz);
            acc2 += wq * mut * dv * dv;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc0 += __shfl_down_sync(0xffffffffu, acc0, o);
        acc1 += __shfl_down_sync(0xffffffffu, acc1, o);
        acc2 += __shfl_down_sync(0xffffffffu, acc2, o);
    }
    if ((t & 31) == 0) {
        red[0][t >> 5] = acc0;
        red[1][t >> 5] = acc1;
        red[2][t >> 5] = acc2;
    }
    __syncthreads();
    if (t < 3) {
        double s = 0;
        for (int w = 0; w < 4; ++w) s += red[t][w];
        partials[blockIdx.x * 3 + t] = s;
    }
}

// Fixed-order sum of the per-block partial triples (deterministic).
__global__ void sum_partials_kernel(const double* __restrict__ partials, int nblocks,
                                    double* __restrict__ out) {
    __shared__ double red[3][256];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        s0 += partials[3 * b];
        s1 += partials[3 * b + 1];
        s2 += partials[3 * b + 2];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

namespace sllbm {

// 1: generic tile kernel, 2: TMA-fed persistent kernel, 0: the requested kernel cannot run.
// The automatic choice takes the TMA-fed kernel where it can run and the mesh (a slab: its
// interior) has enough nodes for its persistent CTAs to run full: on smaller meshes its set-up
// per CTA and the source boxes that wrap around the periodic boundary (all of them on the
// smallest meshes, several images each) make it slower than the generic kernel (measured on
// GB300, FP32 and FP16 storage, time TMA / generic: p = 2 1.05 at 64^3 nodes and 0.81 at 96^3;
// p = 3 1.19 at 96^3, 1.00 at 132^3, 0.92 at 192^3; p = 4 1.03 at 96^3, 0.87 at 128^3; up to
// 3-6x on meshes of a few tiles).  And not for 16-bit storage at p = 3 on an ordinary periodic
// context: there its 6x9x3-node tiles (27 of 32 lanes), the widening of every stored pair and
// the two periodic images of the boxes that wrap around along z leave it 9-18 % slower than
// the generic kernel with two CTAs per SM even at 192^3 nodes, while on a slab (whose boxes
// never wrap along z, e.g. the whole mesh with ghost planes) it is 6 % faster there.
int choose_step_kernel(const sllbm_ctx* c) {
    const bool tma_ok = tma_step_eligible(c);
    if (c->prm.kernel == 2) return tma_ok ? 2 : 0;
    if (c->prm.kernel == 1) return 1;
    const bool dev16 = c->prm.storage == SLLBM_F16DEV || c->prm.storage == SLLBM_BF16DEV;
    const double nodes = static_cast<double>(c->N[0]) * c->N[1] * (static_cast<double>(c->cells[2]) * c->p);
    const double min_nodes = c->p == 2 ? 5e5 : (c->p == 3 ? 3e6 : 1.5e6);
    // (with the Prandtl term the TMA-fed kernel is at best as fast as the generic one: at
    // 128^3 nodes, p = 4, 1.35 ms against 1.36 with ghost planes, 1.51 against 1.35 on the
    // ordinary periodic context; at 192^3, p = 3, 5.28 against 4.25)
    // Compensated moment sums cost the TMA-fed kernel +22 to +52 % (its four epilogue warps
    // issue them) and the generic one +10 to +18 %: the generic kernel is then the faster at
    // p = 3 (192^3 nodes: FP32 4.01 against 4.33 ms) and about as fast with 16-bit storage at
    // p = 4 on the ordinary periodic context (128^3: FP16 1.31 against 1.34 ms, BF16 1.33
    // against 1.31).
    const bool comp_generic = c->compensated && (c->p == 3 || (dev16 && c->p == 4 && !c->slab));
    return (tma_ok && nodes >= min_nodes && !c->prm.pr_correction && !(dev16 && c->p == 3 && !c->slab) &&
            !comp_generic)
               ? 2
               : 1;
}

}  // namespace sllbm

namespace {


int launch_init(sllbm_ctx* ctx, int mode, const double* rho, const double* u, const double* T) {
    int rc = ensure_buffers(ctx);
    if (rc != SLLBM_OK) return rc;
    const int block = 256;
    const unsigned grid = grid_for(ctx->nn, block);
    const double gfac = 2.0 / (ctx->prm.gamma - 1.0) - 3.0;
    const double U0 = ctx->U0, rho0 = ctx->prm.rho0, T0 = ctx->prm.T0, C = ctx->tgv_C;
    void* dst = ctx->buf[ctx->cur];
    with_storage(ctx, [&](auto tag) {
        using S = decltype(tag);
        init_eq_kernel<S><<<grid, block, 0, ctx->stream>>>(
            static_cast<S*>(dst), ctx->nn, ctx->N[0], ctx->N[1], ctx->d_coords[0], ctx->d_coords[1],
            ctx->d_coords[2], mode, U0, rho0, T0, C, rho, u, T, gfac, pop_ref(ctx), vel_const(ctx));
    });
    ctx->launches += 1;
    CK(ctx, cudaGetLastError());
    ctx->initialised = true;
    ctx->steps = 0;
    return SLLBM_OK;
}

// The planes the diagnostics wrap around in, and where they start in the buffer (a slab that
// spans the whole mesh: its interior, above the ghost planes).
int diag_planes(const sllbm_ctx* ctx) { return ctx->slab ? ctx->cells[2] * ctx->p : ctx->N[2]; }
int diag_zoff(const sllbm_ctx* ctx) { return ctx->slab ? ctx->ghost * ctx->p : 0; }

template <int P>
int launch_diag_p(sllbm_ctx* ctx, const void* pop, double* d_out) {
    const long long ncell = static_cast<long long>(ctx->cells[0]) * ctx->cells[1] * ctx->cells[2];
    DiagConst dc;
    std::memcpy(dc.xi, ctx->xi, sizeof(dc.xi));
    std::memcpy(dc.w, ctx->w, sizeof(dc.w));
    dc.ref = pop_ref(ctx);
    double W[kMaxP + 1];
    clenshaw_curtis(P, W);
    for (int j = 0; j <= kMaxP; ++j) dc.W[j] = j <= P ? W[j] : 0.0;
    double D[kMaxP + 1][kMaxP + 1];
    diff_matrix(P, D);
    for (int a = 0; a <= kMaxP; ++a)
        for (int j = 0; j <= kMaxP; ++j) dc.D[a][j] = (a <= P && j <= P) ? D[a][j] : 0.0;
    const double inv_2cv = 0.5 * (ctx->prm.gamma - 1.0);
    const int nb = ctx->partial_blocks;
    with_storage(ctx, [&](auto tag) {
        using S = decltype(tag);
        diag_kernel<S, P><<<nb, 128, 0, ctx->stream>>>(
            static_cast<const S*>(pop), ctx->nn, ctx->N[0], ctx->N[1], diag_planes(ctx), diag_zoff(ctx),
            ctx->cells[0], ctx->cells[1], ncell, inv_2cv, ctx->h[0], ctx->h[1], ctx->h[2], dc, ctx->d_partials);
    });
    sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(ctx->d_partials, nb, d_out);
    ctx->launches += 2;
    CK(ctx, cudaGetLastError());
    return SLLBM_OK;
}

// ---------------------------------------------------------------- diagnostics without allocation
// Scratch of sllbm_diag_noalloc: one partial triple per cell plus the three totals, in a
// file-scope device array (every GPU that loads the library holds these 1.5 MB until exit).
constexpr long long kNoAllocDiagMaxCells = 65536;
static __device__ __align__(256) double g_diag_scratch[3 * kNoAllocDiagMaxCells + 3];

// (Host code cannot use g_diag_scratch's name as a device address: each context looks the
// address up with cudaGetSymbolAddress when it is created, with its device current, and
// keeps it in sllbm_ctx::diag_scratch.  A context created after a cudaDeviceReset, or in
// another CUDA context, thus gets the address of the array as loaded there.)

template <int P>
int launch_diag_cells_into(sllbm_ctx* ctx, const void* pop, double* partials, double* d_out) {
    const long long ncell = static_cast<long long>(ctx->cells[0]) * ctx->cells[1] * ctx->cells[2];
    DiagConst dc;
    std::memcpy(dc.xi, ctx->xi, sizeof(dc.xi));
    std::memcpy(dc.w, ctx->w, sizeof(dc.w));
    dc.ref = pop_ref(ctx);
    double W[kMaxP + 1];
    clenshaw_curtis(P, W);
    for (int j = 0; j <= kMaxP; ++j) dc.W[j] = j <= P ? W[j] : 0.0;
    double D[kMaxP + 1][kMaxP + 1];
    diff_matrix(P, D);
    for (int a = 0; a <= kMaxP; ++a)
        for (int j = 0; j <= kMaxP; ++j) dc.D[a][j] = (a <= P && j <= P) ? D[a][j] : 0.0;
    const double inv_2cv = 0.5 * (ctx->prm.gamma - 1.0);
    const int nb = static_cast<int>(ncell);  // one block, hence one partial triple, per cell
    with_storage(ctx, [&](auto tag) {
        using S = decltype(tag);
        diag_kernel<S, P><<<nb, 128, 0, ctx->stream>>>(
            static_cast<const S*>(pop), ctx->nn, ctx->N[0], ctx->N[1], diag_planes(ctx), diag_zoff(ctx),
            ctx->cells[0], ctx->cells[1], ncell, inv_2cv, ctx->h[0], ctx->h[1], ctx->h[2], dc, partials);
    });
    sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(partials, nb, d_out);
    ctx->launches += 2;
    CK(ctx, cudaGetLastError());
    return SLLBM_OK;
}

}  // namespace

namespace sllbm {

int ensure_buffers(sllbm_ctx* ctx) {
    if (ctx->buf[0] != nullptr) return SLLBM_OK;
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = dev_alloc(&ctx->buf[b], ctx->pop_bytes);
        if (e != cudaSuccess) {
            ctx->last_err = static_cast<int>(e);
            return SLLBM_ENOMEM;
        }
    }
    ctx->own_buf = true;
    ctx->cur = 0;
    return SLLBM_OK;
}

// The step kernel(s) from buf[cur] into buf[1-cur], without the swap.
int launch_current(sllbm_ctx* ctx) {
    const void* src = ctx->buf[ctx->cur];
    void* dst = ctx->buf[1 - ctx->cur];
    return ctx->prm.storage == SLLBM_F64   ? launch_step_f64(ctx, src, dst)
           : ctx->prm.storage == SLLBM_F32 ? launch_step_f32(ctx, src, dst)
                                           : launch_step_f16(ctx, src, dst);
}

int step_launch(sllbm_ctx* ctx) {
    if (ctx->slab && ctx->cells[2] == ctx->z_cells_global) {
        // a slab spanning the whole mesh is periodic along z by its own ghost planes: refresh
        // them from the opposite end of the interior before the step reads them
        const int rc = sllbm_halo_periodic(ctx, nullptr);
        if (rc != SLLBM_OK) return rc;
    }
    const int rc = launch_current(ctx);
    if (rc != SLLBM_OK) return rc;
    ctx->cur = 1 - ctx->cur;
    ++ctx->steps;
    return SLLBM_OK;
}

void fill_step_args(const sllbm_ctx* ctx, const void* src, void* dst, StepArgs* a) {
    a->src = src;
    a->dst = dst;
    for (int d = 0; d < 3; ++d) {
        a->N[d] = ctx->N[d];
        a->cells[d] = ctx->cells[d];
        a->tiles[d] = 1;
    }
    a->nn = ctx->nn;
    a->mu_over_dt = ctx->mu_inf / ctx->dt;
    const double cv = 1.0 / (ctx->prm.gamma - 1.0);
    a->inv_2cv = 0.5 / cv;
    a->gfac = 2.0 * cv - 3.0;
    a->inv_pr = 1.0 / ctx->prm.Pr;
    a->pr = ctx->prm.pr_correction;
    a->rho0 = ctx->prm.rho0;
    a->T0 = ctx->prm.T0;
    a->collide = ctx->prm.collide;
    a->flag = ctx->prm.nonfinite_check ? ctx->d_flag : nullptr;
    a->flag_err = ctx->d_flag + 1;
    a->abort_req = ctx->d_flag + 2;
    a->wait_ns = ctx->wait_ns;
    a->z0 = ctx->ghost;
    a->tz_begin = 0;
}

}  // namespace sllbm

extern "C" {

void sllbm_default_params(sllbm_params* p) {
    if (p == nullptr) return;
    std::memset(p, 0, sizeof(*p));
    p->Ma = 0.5;
    p->Re = 1600.0;
    p->Pr = 0.7;
    p->gamma = 1.4;
    p->T0 = 1.0;
    p->rho0 = 1.0;
    p->dt_or_courant = 1.0;
    p->dt_is_courant = 1;
    p->pr_correction = 0;
    p->storage = SLLBM_F32;
    p->nonfinite_check = 0;
    p->tgv_C = -1.0;
    p->mu_inf_override = 0.0;
    p->collide = 1;
    p->kernel = 0;
}

}  // extern "C"

namespace {

// sllbm_create (slab = 0: the whole periodic mesh) and sllbm_create_slab (slab = 1: the
// z-cells [z_begin, z_begin + z_cells) with ghost cells of halo on both sides).
int create_ctx(const sllbm_mesh* mesh, int p, sllbm_velset vs, const sllbm_params* prm, int slab, int z_begin,
               int z_cells, void* cuda_stream, sllbm_ctx** out) {
    if (out == nullptr) return SLLBM_EINVAL;
    *out = nullptr;
    if (mesh == nullptr || prm == nullptr || vs != SLLBM_D3Q45) return SLLBM_EINVAL;
    if (p < 2 || p > 4) return SLLBM_EINVAL;
    if (prm->storage != SLLBM_F64 && prm->storage != SLLBM_F32 && prm->storage != SLLBM_F16DEV &&
        prm->storage != SLLBM_BF16DEV)
        return SLLBM_EINVAL;
    if (!(prm->gamma > 1.0) || !(prm->Pr > 0.0) || !(prm->T0 > 0.0) || !(prm->rho0 > 0.0))
        return SLLBM_EINVAL;
    if (!(prm->dt_or_courant > 0.0)) return SLLBM_EINVAL;
    long long nn = 1;
    for (int d = 0; d < 3; ++d) {
        if (mesh->cells[d] < 1 || !(mesh->L[d] > 0.0)) return SLLBM_EINVAL;
        if (static_cast<long long>(mesh->cells[d]) * p > (1 << 20)) return SLLBM_EINVAL;
        nn *= static_cast<long long>(mesh->cells[d]) * p;
    }
    if (nn > 0x7fffffffLL) return SLLBM_EINVAL;  // per-field offsets are 32-bit
    if (slab && (z_begin < 0 || z_begin >= mesh->cells[2] || z_cells < 1 || z_cells > mesh->cells[2]))
        return SLLBM_EINVAL;
    sllbm_ctx* c = static_cast<sllbm_ctx*>(std::calloc(1, sizeof(sllbm_ctx)));
    if (c == nullptr) return SLLBM_ENOMEM;
    c->p = p;
    c->prm = *prm;
    c->nn = nn;
    for (int d = 0; d < 3; ++d) {
        c->cells[d] = mesh->cells[d];
        c->N[d] = mesh->cells[d] * p;
        c->L[d] = mesh->L[d];
        c->h[d] = mesh->L[d] / mesh->cells[d];
    }
    c->z_cells_global = mesh->cells[2];
    build_velocity_set(c->xi, c->w);
    double mx = 0.0;
    for (int i = 0; i < kQ; ++i)
        mx = std::fmax(mx, std::sqrt(c->xi[i][0] * c->xi[i][0] + c->xi[i][1] * c->xi[i][1]
                                     + c->xi[i][2] * c->xi[i][2]));
    c->max_xi = mx;
    if (prm->dt_is_courant) {
        double dxn = c->L[0] / c->N[0];
        for (int d = 1; d < 3; ++d) dxn = std::fmin(dxn, c->L[d] / c->N[d]);
        c->dt = prm->dt_or_courant * dxn / mx;
    } else {
        c->dt = prm->dt_or_courant;
    }
    c->U0 = prm->Ma * std::sqrt(prm->gamma * prm->T0);
    c->mu_inf = prm->mu_inf_override > 0.0 ? prm->mu_inf_override : prm->rho0 * c->U0 / prm->Re;
    c->tgv_C = prm->tgv_C < 0.0 ? prm->gamma * prm->Ma * prm->Ma : prm->tgv_C;
    if (!(c->mu_inf > 0.0) && prm->collide) {
        std::free(c);
        return SLLBM_EINVAL;
    }
    c->max_shift = 0;
    bool span_ok = true;
    for (int d = 0; d < 3; ++d) {
        build_dir_table(p, c->h[d], c->dt, c->xi, d, &c->dir[d]);
        for (int i = 0; i < kQ; ++i) {
            int lo = c->dir[d].shift[i][0], hi = lo;
            for (int a = 0; a < p; ++a) {
                int k = c->dir[d].shift[i][a];
                int s = std::abs(k);
                if (s > c->max_shift) c->max_shift = s;
                lo = k < lo ? k : lo;
                hi = k > hi ? k : hi;
            }
            // the departure points of one cell's nodes span less than a cell, so at most
            // two neighbouring cells; the kernel's source-box sizes rely on this
            if (hi - lo > 1) span_ok = false;
        }
    }
    if (c->max_shift > 100 || !span_ok) {
        std::free(c);
        return SLLBM_EINVAL;
    }
    if (slab) {
        // Ghost cells per side: a tile's source box starts kmin >= -max_shift cells below the
        // tile and ends with the first node of the cell kmin + span <= max_shift cells above
        // its last cell, so max_shift + 1 cells on each side hold every source node, and the
        // halo of one side comes from one neighbouring slab if the slab has at least as many
        // cells.
        c->slab = 1;
        c->z_begin = z_begin;
        c->ghost = c->max_shift + 1;
        if (z_cells < c->ghost) {
            std::free(c);
            return SLLBM_EINVAL;
        }
        c->cells[2] = z_cells;
        c->N[2] = (z_cells + 2 * c->ghost) * p;
        c->nn = static_cast<long long>(c->N[0]) * c->N[1] * c->N[2];
        if (c->nn > 0x7fffffffLL) {
            std::free(c);
            return SLLBM_EINVAL;
        }
        nn = c->nn;
    }
    c->elem = prm->storage == SLLBM_F64 ? sizeof(double) : prm->storage == SLLBM_F32 ? sizeof(float) : 2;
    c->pop_bytes = static_cast<size_t>(2 * kQ) * static_cast<size_t>(nn) * c->elem;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->wait_ns = kDefaultWaitNs;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) {
        for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
            e = dev_alloc(&c->d_coords[d], sizeof(double) * c->N[d]);
            if (e != cudaSuccess) break;
            double* x = static_cast<double*>(std::malloc(sizeof(double) * c->N[d]));
            if (x == nullptr) {
                e = cudaErrorMemoryAllocation;
                break;
            }
            // (a slab's local planes start `ghost` cells below its first interior cell; their
            // cells are numbered on the whole periodic mesh)
            const int c_first = d == 2 ? c->z_begin - c->ghost : 0;
            const int c_wrap = d == 2 ? c->z_cells_global : c->cells[d];
            for (int cc = 0; cc < c->N[d] / p; ++cc) {
                const int gc = ((c_first + cc) % c_wrap + c_wrap) % c_wrap;
                for (int a = 0; a < p; ++a)
                    x[cc * p + a] = gc * c->h[d] + (1.0 - std::cos(kPi * a / p)) * 0.5 * c->h[d];
            }
            e = cudaMemcpy(c->d_coords[d], x, sizeof(double) * c->N[d], cudaMemcpyHostToDevice);
            std::free(x);
        }
        // d_flag[0]: non-finite rho/T seen; d_flag[1]: a bounded device wait gave up (2) or the
        // kernel honoured an abort request (4); d_flag[2]: the abort request
        if (e == cudaSuccess) e = dev_alloc(&c->d_flag, 3 * sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(c->d_flag, 0, 3 * sizeof(int));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->ctl_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
        // the device address of sllbm_diag_noalloc's static scratch on this device
        if (e == cudaSuccess) {
            void* addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_diag_scratch);
            c->diag_scratch = static_cast<double*>(addr);
        }
    }
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? SLLBM_ENOMEM : SLLBM_ECUDA;
        sllbm_destroy(c);
        return code;
    }
    c->step_kernel = choose_step_kernel(c);
    if (c->step_kernel == 0) {  // the TMA kernel was requested but cannot run this case
        sllbm_destroy(c);
        return SLLBM_EINVAL;
    }
    *out = c;
    return SLLBM_OK;
}

// Per velocity: the first state plane of its chunk and its plane count, and the chunk's
// offset in the packed halo buffer (4-byte words; a plane of (f, g) pairs is a whole number
// of words).
struct HaloMap {
    int plane0[kQ];
    int planes[kQ];
    long long packed_word[kQ];
};

// Copies each velocity's chunk of planes between the state and the packed halo buffer
// (to_state: packed -> state); blockIdx.y is the velocity.
__global__ void __launch_bounds__(256) halo_copy_kernel(unsigned* __restrict__ state, unsigned* __restrict__ halo,
                                                         long long plane_words, long long vstride_words,
                                                         int to_state, const __grid_constant__ HaloMap m) {
    const int i = blockIdx.y;
    const long long n = static_cast<long long>(m.planes[i]) * plane_words;
    unsigned* sp = state + i * vstride_words + static_cast<long long>(m.plane0[i]) * plane_words;
    unsigned* hp = halo + m.packed_word[i];
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (to_state) sp[k] = hp[k];
        else hp[k] = sp[k];
    }
}

// Planes of velocity i in the ghost region on `side` that the step reads (0 below, 1
// above), from its departure cell shifts along z: a tile's source box starts kmin cells
// below its first cell and ends with the first node of the cell kmin + span + 1 above its
// last one, so below the slab it reads -kmin cells (when kmin < 0) and above it
// (kmin + span) cells plus one plane (when kmin + span >= 0).
int ghost_planes(const sllbm_ctx* c, int i, int side) {
    int kmn = 1 << 20, kmx = -(1 << 20);
    for (int a = 0; a < c->p; ++a) {
        const int k = c->dir[2].shift[i][a];
        kmn = k < kmn ? k : kmn;
        kmx = k > kmx ? k : kmx;
    }
    if (side == 0) return kmn < 0 ? -kmn * c->p : 0;
    return kmx >= 0 ? kmx * c->p + 1 : 0;
}

// A slab that spans the whole mesh along z is its own neighbour: each velocity's ghost planes
// below it are its highest interior planes and those above it its lowest ones.  One launch
// copies both sides inside the state buffer (blockIdx.z = side, blockIdx.y = velocity), in
// 16-byte words when a plane is a whole number of them (else 4-byte words).
struct PeriodicMap {
    int dst0[2][kQ];  // first ghost plane written
    int src0[2][kQ];  // first interior plane read
    int planes[2][kQ];
};

template <typename W>
__global__ void __launch_bounds__(256) halo_periodic_kernel(W* __restrict__ state, long long plane_words,
                                                             long long vstride_words, const __grid_constant__ PeriodicMap m) {
    const int side = blockIdx.z, i = blockIdx.y;
    const long long n = static_cast<long long>(m.planes[side][i]) * plane_words;
    W* base = state + i * vstride_words;
    const W* src = base + static_cast<long long>(m.src0[side][i]) * plane_words;
    W* dst = base + static_cast<long long>(m.dst0[side][i]) * plane_words;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<long long>(gridDim.x) * blockDim.x)
        dst[k] = src[k];
}

// Bytes of the packed halo sllbm_halo_pack(side) writes (the receiving slab's ghost region
// on the other side).
size_t halo_pack_bytes(const sllbm_ctx* c, int side) {
    const size_t plane_bytes = static_cast<size_t>(c->N[0]) * c->N[1] * 2 * c->elem;
    size_t planes = 0;
    for (int i = 0; i < kQ; ++i) planes += static_cast<size_t>(ghost_planes(c, i, 1 - side));
    return planes * plane_bytes;
}

// Packing (to_state = 0) copies, per velocity, the interior planes next to `side` that the
// neighbouring slab on that side reads as its ghost planes; unpacking (to_state = 1) writes a
// neighbour's packed planes into this slab's ghost planes on `side` -- only the planes each
// velocity's source boxes reach, not the whole ghost width.
int halo_copy(sllbm_ctx* ctx, int side, void* halo, int to_state, cudaStream_t stream) {
    if (ctx == nullptr || !ctx->slab || halo == nullptr || (side != 0 && side != 1)) return SLLBM_EINVAL;
    if (ctx->buf[ctx->cur] == nullptr) return SLLBM_EINVAL;
    const int gp = ctx->ghost * ctx->p;
    const int top = gp + ctx->cells[2] * ctx->p;  // first plane above the interior
    const long long plane_words = static_cast<long long>(ctx->N[0]) * ctx->N[1] * 2 * ctx->elem / 4;
    HaloMap m;
    long long off = 0;
    int most = 0;
    for (int i = 0; i < kQ; ++i) {
        // pack(side) serves the neighbour's ghost region on the other side; unpack(side)
        // fills this slab's ghost region on `side`
        const int n = ghost_planes(ctx, i, to_state ? side : 1 - side);
        m.planes[i] = n;
        m.plane0[i] = to_state ? (side == 0 ? gp - n : top) : (side == 0 ? gp : top - n);
        m.packed_word[i] = off;
        off += static_cast<long long>(n) * plane_words;
        most = n > most ? n : most;
    }
    if (most == 0) return SLLBM_OK;
    const long long per = static_cast<long long>(most) * plane_words;
    long long bx = (per + 255) / 256;
    if (bx > 1024) bx = 1024;
    halo_copy_kernel<<<dim3(static_cast<unsigned>(bx), kQ), 256, 0, stream>>>(
        static_cast<unsigned*>(ctx->buf[ctx->cur]), static_cast<unsigned*>(halo), plane_words,
        static_cast<long long>(ctx->N[2]) * plane_words, to_state, m);
    ctx->launches += 1;
    CK(ctx, cudaGetLastError());
    return SLLBM_OK;
}

}  // namespace

extern "C" {

int sllbm_create(const sllbm_mesh* mesh, int p, sllbm_velset vs, const sllbm_params* prm,
                 void* cuda_stream, sllbm_ctx** out) {
    return create_ctx(mesh, p, vs, prm, 0, 0, 0, cuda_stream, out);
}

int sllbm_create_slab(const sllbm_mesh* mesh, int p, sllbm_velset vs, const sllbm_params* prm, int z_begin,
                      int z_cells, void* cuda_stream, sllbm_ctx** out) {
    return create_ctx(mesh, p, vs, prm, 1, z_begin, z_cells, cuda_stream, out);
}

int sllbm_slab_info(const sllbm_ctx* ctx, int* ghost_cells, size_t* halo_bytes) {
    if (ctx == nullptr || !ctx->slab) return SLLBM_EINVAL;
    if (ghost_cells != nullptr) *ghost_cells = ctx->ghost;
    if (halo_bytes != nullptr) {
        const size_t b0 = halo_pack_bytes(ctx, 0), b1 = halo_pack_bytes(ctx, 1);
        *halo_bytes = b0 > b1 ? b0 : b1;
    }
    return SLLBM_OK;
}

int sllbm_slab_halo_bytes(const sllbm_ctx* ctx, int side, size_t* bytes) {
    if (ctx == nullptr || !ctx->slab || (side != 0 && side != 1) || bytes == nullptr) return SLLBM_EINVAL;
    *bytes = halo_pack_bytes(ctx, side);
    return SLLBM_OK;
}

int sllbm_halo_pack(sllbm_ctx* ctx, int side, void* halo, void* cuda_stream) {
    NvtxRange range("sllbm_halo_pack");
    if (ctx == nullptr) return SLLBM_EINVAL;
    return halo_copy(ctx, side, halo, 0, cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream);
}

int sllbm_halo_unpack(sllbm_ctx* ctx, int side, const void* halo, void* cuda_stream) {
    NvtxRange range("sllbm_halo_unpack");
    if (ctx == nullptr) return SLLBM_EINVAL;
    return halo_copy(ctx, side, const_cast<void*>(halo), 1,
                     cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream);
}

int sllbm_halo_periodic(sllbm_ctx* ctx, void* cuda_stream) {
    if (ctx == nullptr || !ctx->slab || ctx->cells[2] != ctx->z_cells_global) return SLLBM_EINVAL;
    if (ctx->buf[ctx->cur] == nullptr) return SLLBM_EINVAL;
    const cudaStream_t stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
    const int gp = ctx->ghost * ctx->p;
    const int top = gp + ctx->cells[2] * ctx->p;
    PeriodicMap m;
    int most = 0;
    for (int i = 0; i < kQ; ++i) {
        const int nb = ghost_planes(ctx, i, 0), na = ghost_planes(ctx, i, 1);
        m.planes[0][i] = nb;  // below: the highest interior planes
        m.dst0[0][i] = gp - nb;
        m.src0[0][i] = top - nb;
        m.planes[1][i] = na;  // above: the lowest interior planes
        m.dst0[1][i] = top;
        m.src0[1][i] = gp;
        most = nb > most ? nb : most;
        most = na > most ? na : most;
    }
    if (most == 0) return SLLBM_OK;
    const size_t plane_bytes = static_cast<size_t>(ctx->N[0]) * ctx->N[1] * 2 * ctx->elem;
    const bool w16 = plane_bytes % 16 == 0;
    const long long plane_words = static_cast<long long>(plane_bytes / (w16 ? 16 : 4));
    const long long per = static_cast<long long>(most) * plane_words;
    long long bx = (per + 255) / 256;
    if (bx > 512) bx = 512;
    const dim3 grid(static_cast<unsigned>(bx), kQ, 2);
    if (w16)
        halo_periodic_kernel<uint4><<<grid, 256, 0, stream>>>(static_cast<uint4*>(ctx->buf[ctx->cur]), plane_words,
                                                             static_cast<long long>(ctx->N[2]) * plane_words, m);
    else
        halo_periodic_kernel<unsigned><<<grid, 256, 0, stream>>>(static_cast<unsigned*>(ctx->buf[ctx->cur]),
                                                                plane_words,
                                                                static_cast<long long>(ctx->N[2]) * plane_words, m);
    ctx->launches += 1;
    CK(ctx, cudaGetLastError());
    return SLLBM_OK;
}

int sllbm_step_begin(sllbm_ctx* ctx) {
    NvtxRange range("sllbm_step_begin");
    if (ctx == nullptr || !ctx->slab) return SLLBM_EINVAL;
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    if (ctx->prm.nonfinite_check) CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    if (ctx->cells[2] == ctx->z_cells_global) {  // periodic by its own ghost planes (see step_launch)
        const int rc0 = sllbm_halo_periodic(ctx, nullptr);
        if (rc0 != SLLBM_OK) return rc0;
    }
    ctx->region = 1;
    const int rc = launch_current(ctx);
    ctx->region = 0;
    return rc;
}

int sllbm_step_end(sllbm_ctx* ctx) {
    NvtxRange range("sllbm_step_end");
    if (ctx == nullptr || !ctx->slab) return SLLBM_EINVAL;
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    ctx->region = 2;
    const int rc = launch_current(ctx);
    ctx->region = 0;
    if (rc != SLLBM_OK) return rc;
    ctx->cur = 1 - ctx->cur;
    ++ctx->steps;
    if (ctx->prm.nonfinite_check) {
        int flags[2] = {0, 0};
        CK(ctx, cudaMemcpyAsync(flags, ctx->d_flag, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        if (flags[1]) {
            CK(ctx, cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), ctx->stream));
            return (flags[1] & 2) ? SLLBM_ETIMEOUT : SLLBM_EABORTED;
        }
        if (flags[0]) return SLLBM_ENONFINITE;
    }
    return SLLBM_OK;
}

void sllbm_destroy(sllbm_ctx* ctx) {
    if (ctx == nullptr) return;
    if (ctx->own_buf) {
        cudaFree(ctx->buf[0]);
        cudaFree(ctx->buf[1]);
    }
    for (int d = 0; d < 3; ++d) cudaFree(ctx->d_coords[d]);
    cudaFree(ctx->d_flag);
    if (ctx->ctl_stream) cudaStreamDestroy(ctx->ctl_stream);
    cudaFree(ctx->d_partials);
    adjoint_release(ctx);
    for (int b = 0; b < 6; ++b) cudaFree(ctx->pipe_buf[b]);
    for (int s = 0; s < 2; ++s)
        if (ctx->pipe_stream[s]) cudaStreamDestroy(ctx->pipe_stream[s]);
    for (int e = 0; e < 9; ++e)
        if (ctx->pipe_ev[e]) cudaEventDestroy(ctx->pipe_ev[e]);
    std::free(ctx->step_blob);
    std::free(ctx);
}

int sllbm_get_info(const sllbm_ctx* ctx, sllbm_info_t* info) {
    if (ctx == nullptr || info == nullptr) return SLLBM_EINVAL;
    for (int d = 0; d < 3; ++d) info->N[d] = ctx->N[d];
    info->p = ctx->p;
    info->nodes = ctx->nn;
    info->Q = kQ;
    info->dt = ctx->dt;
    info->U0 = ctx->U0;
    info->mu_inf = ctx->mu_inf;
    info->max_xi = ctx->max_xi;
    info->pop_bytes = ctx->pop_bytes;
    info->storage = ctx->prm.storage;
    info->max_cell_shift = ctx->max_shift;
    info->step_kernel = ctx->step_kernel;
    info->step_variant = ctx->step_kernel == 2 ? 0 : 1 + ctx->tile_shape;
    return SLLBM_OK;
}

int sllbm_velset_table(const sllbm_ctx* ctx, double* xi, double* w) {
    if (ctx == nullptr || xi == nullptr || w == nullptr) return SLLBM_EINVAL;
    std::memcpy(xi, ctx->xi, sizeof(ctx->xi));
    std::memcpy(w, ctx->w, sizeof(ctx->w));
    return SLLBM_OK;
}

int sllbm_set_buffers(sllbm_ctx* ctx, void* popA, void* popB, size_t bytes) {
    if (ctx == nullptr || popA == nullptr || popB == nullptr || popA == popB) return SLLBM_EINVAL;
    if (bytes < ctx->pop_bytes) return SLLBM_EINVAL;
    if (ctx->own_buf) {
        cudaFree(ctx->buf[0]);
        cudaFree(ctx->buf[1]);
        ctx->own_buf = false;
    }
    ctx->buf[0] = popA;
    ctx->buf[1] = popB;
    ctx->cur = 0;
    ctx->initialised = false;
    ctx->tmap_src[0] = ctx->tmap_src[1] = nullptr;  // TMA descriptors describe old buffers
    return SLLBM_OK;
}

void* sllbm_current_buffer(const sllbm_ctx* ctx) {
    if (ctx == nullptr || !ctx->initialised) return nullptr;
    return ctx->buf[ctx->cur];
}

int sllbm_init_tgv(sllbm_ctx* ctx) {
    if (ctx == nullptr) return SLLBM_EINVAL;
    return launch_init(ctx, 0, nullptr, nullptr, nullptr);
}

int sllbm_init_fields(sllbm_ctx* ctx, const double* rho, const double* u, const double* T,
                      int on_device) {
    if (ctx == nullptr || rho == nullptr || u == nullptr || T == nullptr) return SLLBM_EINVAL;
    if (on_device) return launch_init(ctx, 1, rho, u, T);
    double* d = nullptr;
    const size_t nb = sizeof(double) * static_cast<size_t>(ctx->nn);
    cudaError_t e = dev_alloc(&d, 5 * nb);
    if (e != cudaSuccess) {
        ctx->last_err = static_cast<int>(e);
        return SLLBM_ENOMEM;
    }
    int rc = SLLBM_OK;
    e = cudaMemcpyAsync(d, rho, nb, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + ctx->nn, u, 3 * nb, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 4 * ctx->nn, T, nb, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        rc = launch_init(ctx, 1, d, d + ctx->nn, d + 4 * ctx->nn);
        if (rc == SLLBM_OK) e = cudaStreamSynchronize(ctx->stream);
    }
    cudaFree(d);
    if (e != cudaSuccess) return fail(ctx, e);
    return rc;
}

int sllbm_set_populations(sllbm_ctx* ctx, const double* pop, int on_device) {
    if (ctx == nullptr || pop == nullptr) return SLLBM_EINVAL;
    int rc = ensure_buffers(ctx);
    if (rc != SLLBM_OK) return rc;
    const long long count = 2LL * kQ * ctx->nn;
    void* dst = ctx->buf[ctx->cur];
    const double* src = pop;
    double* tmp = nullptr;
    if (!on_device) {
        CK(ctx, dev_alloc(&tmp, count * sizeof(double)));
        cudaError_t e = cudaMemcpyAsync(tmp, pop, count * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return fail(ctx, e);
        }
        src = tmp;
    }
    with_storage(ctx, [&](auto tag) {
        using S = decltype(tag);
        pack_kernel<S><<<grid_for(count, 256), 256, 0, ctx->stream>>>(src, static_cast<S*>(dst), ctx->nn, pop_ref(ctx),
                                                                       vel_const(ctx));
    });
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (tmp != nullptr) {
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(tmp);
    }
    if (e != cudaSuccess) return fail(ctx, e);
    ctx->initialised = true;
    ctx->steps = 0;
    return SLLBM_OK;
}

int sllbm_get_populations(sllbm_ctx* ctx, double* pop, int on_device) {
    if (ctx == nullptr || pop == nullptr) return SLLBM_EINVAL;
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    const long long count = 2LL * kQ * ctx->nn;
    const void* src = ctx->buf[ctx->cur];
    double* dst = pop;
    double* tmp = nullptr;
    if (!on_device) {
        CK(ctx, dev_alloc(&tmp, count * sizeof(double)));
        dst = tmp;
    }
    with_storage(ctx, [&](auto tag) {
        using S = decltype(tag);
        unpack_kernel<S><<<grid_for(count, 256), 256, 0, ctx->stream>>>(static_cast<const S*>(src), dst, ctx->nn,
                                                                         pop_ref(ctx), vel_const(ctx));
    });
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (tmp != nullptr) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(pop, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(tmp);
    }
    if (e != cudaSuccess) return fail(ctx, e);
    return SLLBM_OK;
}

int sllbm_step(sllbm_ctx* ctx, int n) {
    NvtxRange range("sllbm_step");
    if (ctx == nullptr || n < 0) return SLLBM_EINVAL;
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    if (ctx->prm.nonfinite_check) CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    for (int s = 0; s < n; ++s) {
        int rc = step_launch(ctx);
        if (rc != SLLBM_OK) return rc;
    }
    if (ctx->prm.nonfinite_check) {
        int flags[2] = {0, 0};
        CK(ctx, cudaMemcpyAsync(flags, ctx->d_flag, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        if (flags[1]) {
            CK(ctx, cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), ctx->stream));
            return (flags[1] & 2) ? SLLBM_ETIMEOUT : SLLBM_EABORTED;
        }
        if (flags[0]) return SLLBM_ENONFINITE;
    }
    return SLLBM_OK;
}

int sllbm_load_state(sllbm_ctx* ctx, const void* state) {
    if (ctx == nullptr || state == nullptr) return SLLBM_EINVAL;
    int rc = ensure_buffers(ctx);
    if (rc != SLLBM_OK) return rc;
    if (state != ctx->buf[ctx->cur])
        CK(ctx, cudaMemcpyAsync(ctx->buf[ctx->cur], state, ctx->pop_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->initialised = true;
    ctx->steps = 0;
    return SLLBM_OK;
}

int sllbm_set_mu_inf(sllbm_ctx* ctx, double mu_inf) {
    if (ctx == nullptr || !(mu_inf > 0.0)) return SLLBM_EINVAL;
    ctx->mu_inf = mu_inf;
    return SLLBM_OK;
}

int sllbm_status(sllbm_ctx* ctx) {
    if (ctx == nullptr) return SLLBM_EINVAL;
    int err = 0;
    CK(ctx, cudaMemcpyAsync(&err, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (err) {
        CK(ctx, cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        return (err & 2) ? SLLBM_ETIMEOUT : SLLBM_EABORTED;
    }
    return SLLBM_OK;
}

int sllbm_moments(sllbm_ctx* ctx, double* rho, double* u, double* T, int on_device) {
    if (ctx == nullptr || rho == nullptr || u == nullptr || T == nullptr) return SLLBM_EINVAL;
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    const size_t nb = sizeof(double) * static_cast<size_t>(ctx->nn);
    double* d = nullptr;
    double *dr = rho, *du = u, *dT = T;
    if (!on_device) {
        CK(ctx, dev_alloc(&d, 5 * nb));
        dr = d;
        du = d + ctx->nn;
        dT = d + 4 * ctx->nn;
    }
    const double inv_2cv = 0.5 * (ctx->prm.gamma - 1.0);
    const void* pop = ctx->buf[ctx->cur];
    const unsigned grid = grid_for(ctx->nn, 256);
    with_storage(ctx, [&](auto tag) {
        using S = decltype(tag);
        moments_kernel<S><<<grid, 256, 0, ctx->stream>>>(static_cast<const S*>(pop), ctx->nn, inv_2cv, dr, du, dT,
                                                         pop_ref(ctx), vel_const(ctx));
    });
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (!on_device) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(rho, dr, nb, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, 3 * nb, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(T, dT, nb, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(d);
    }
    if (e != cudaSuccess) return fail(ctx, e);
    return SLLBM_OK;
}

int sllbm_diag(sllbm_ctx* ctx, double* Ek, double* eps_s, double* eps_c) {
    NvtxRange range("sllbm_diag");
    if (ctx == nullptr || Ek == nullptr || eps_s == nullptr || eps_c == nullptr) return SLLBM_EINVAL;
    if (ctx->slab && ctx->cells[2] != ctx->z_cells_global) return SLLBM_EINVAL;  // a part of a mesh
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    if (ctx->d_partials == nullptr) {
        const long long ncell = static_cast<long long>(ctx->cells[0]) * ctx->cells[1] * ctx->cells[2];
        ctx->partial_blocks = static_cast<int>(ncell < 2048 ? ncell : 2048);
        // 3 partial sums per block, then the 3 totals
        cudaError_t e = dev_alloc(&ctx->d_partials, sizeof(double) * (3 * ctx->partial_blocks + 3));
        if (e != cudaSuccess) {
            ctx->d_partials = nullptr;
            ctx->last_err = static_cast<int>(e);
            return SLLBM_ENOMEM;
        }
    }
    double* d_out = ctx->d_partials + 3 * ctx->partial_blocks;
    const void* pop = ctx->buf[ctx->cur];
    int rc = ctx->p == 2 ? launch_diag_p<2>(ctx, pop, d_out)
           : ctx->p == 3 ? launch_diag_p<3>(ctx, pop, d_out)
                         : launch_diag_p<4>(ctx, pop, d_out);
    if (rc != SLLBM_OK) return rc;
    double h[3];
    CK(ctx, cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    const double vol = ctx->L[0] * ctx->L[1] * ctx->L[2];
    const double u2 = ctx->U0 * ctx->U0;
    const double rho0 = ctx->prm.rho0;
    *Ek = h[0] / vol / (rho0 * u2);
    *eps_s = h[1] / vol / (rho0 * ctx->prm.Re * u2);
    *eps_c = 4.0 / 3.0 * h[2] / vol / (rho0 * ctx->prm.Re * u2);
    return SLLBM_OK;
}

// Same results as sllbm_diag (up to summation order) without allocating device memory:
// for callers whose device memory is owned by another allocator or a fixed budget, or
// whose loop must not pay for cudaMalloc/cudaFree (cudaFree synchronises the device).
// The scratch is g_diag_scratch above, at the device address the context looked up when it
// was created (on its device, so nothing here touches the symbol).  All calls share the
// array and each overwrites every entry it reads, so nothing needs clearing, but calls
// that overlap on the GPU (other streams, other contexts) race on it.
int sllbm_diag_noalloc(sllbm_ctx* ctx, double* Ek, double* eps_s, double* eps_c) {
    if (ctx == nullptr || Ek == nullptr || eps_s == nullptr || eps_c == nullptr) return SLLBM_EINVAL;
    if (ctx->slab && ctx->cells[2] != ctx->z_cells_global) return SLLBM_EINVAL;  // a part of a mesh
    if (!ctx->initialised) return SLLBM_ENOTREADY;
    const long long ncell = static_cast<long long>(ctx->cells[0]) * ctx->cells[1] * ctx->cells[2];
    if (ncell > kNoAllocDiagMaxCells) return SLLBM_EINVAL;  // more cells than the static scratch holds
    int dev = 0;
    CK(ctx, cudaGetDevice(&dev));
    if (dev != ctx->device || ctx->diag_scratch == nullptr) return SLLBM_EINVAL;  // not the context's device
    double* scratch = ctx->diag_scratch;
    double* d_out = scratch + 3 * ncell;
    const void* pop = ctx->buf[ctx->cur];
    int rc = ctx->p == 2 ? launch_diag_cells_into<2>(ctx, pop, scratch, d_out)
           : ctx->p == 3 ? launch_diag_cells_into<3>(ctx, pop, scratch, d_out)
                         : launch_diag_cells_into<4>(ctx, pop, scratch, d_out);
    if (rc != SLLBM_OK) return rc;
    double h[3];
    CK(ctx, cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    const double vol = ctx->L[0] * ctx->L[1] * ctx->L[2];
    const double u2 = ctx->U0 * ctx->U0;
    const double rho0 = ctx->prm.rho0;
    *Ek = h[0] / vol / (rho0 * u2);
    *eps_s = h[1] / vol / (rho0 * ctx->prm.Re * u2);
    *eps_c = 4.0 / 3.0 * h[2] / vol / (rho0 * ctx->prm.Re * u2);
    return SLLBM_OK;
}

int sllbm_run_host(sllbm_ctx* ctx, const void* pop_in, void* pop_out, int n) {
    NvtxRange range("sllbm_run_host");
    if (ctx == nullptr || pop_in == nullptr || pop_out == nullptr || n < 0) return SLLBM_EINVAL;
    int rc = ensure_buffers(ctx);
    if (rc != SLLBM_OK) return rc;
    CK(ctx, cudaMemcpyAsync(ctx->buf[ctx->cur], pop_in, ctx->pop_bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->initialised = true;
    ctx->steps = 0;
    rc = sllbm_step(ctx, n);
    if (rc != SLLBM_OK) return rc;
    CK(ctx, cudaMemcpyAsync(pop_out, ctx->buf[ctx->cur], ctx->pop_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

// Pipelined end-to-end runs of independent states: state k uses device slot k % 3 (two
// buffers each, separate from the context's own), its host-to-device copy on one copy
// stream, its steps on the context's stream, its device-to-host copy on the other copy
// stream; events order the three per slot, so that the copies of neighbouring states run
// in both directions at once while a state is stepped.  With three slots the copy of state
// k + 3 into a slot never waits for the copy out of state k (with two it did: 1.2x slower).
int sllbm_run_host_many(sllbm_ctx* ctx, const void* const* pop_in, void* const* pop_out, int count, int n) {
    NvtxRange range("sllbm_run_host_many");
    if (ctx == nullptr || pop_in == nullptr || pop_out == nullptr || count < 1 || n < 0) return SLLBM_EINVAL;
    for (int k = 0; k < count; ++k)
        if (pop_in[k] == nullptr || pop_out[k] == nullptr) return SLLBM_EINVAL;
    if (ctx->pipe_buf[0] == nullptr) {
        for (int b = 0; b < 6; ++b) {
            cudaError_t e = dev_alloc(&ctx->pipe_buf[b], ctx->pop_bytes);
            if (e != cudaSuccess) {
                for (int j = 0; j < b; ++j) cudaFree(ctx->pipe_buf[j]);
                for (int j = 0; j < 6; ++j) ctx->pipe_buf[j] = nullptr;
                ctx->last_err = static_cast<int>(e);
                return SLLBM_ENOMEM;
            }
        }
        for (int s = 0; s < 2; ++s) CK(ctx, cudaStreamCreateWithFlags(&ctx->pipe_stream[s], cudaStreamNonBlocking));
        for (int e = 0; e < 9; ++e) CK(ctx, cudaEventCreateWithFlags(&ctx->pipe_ev[e], cudaEventDisableTiming));
    }
    void* own[2] = {ctx->buf[0], ctx->buf[1]};
    const int own_cur = ctx->cur;
    const bool own_init = ctx->initialised;
    int rc = SLLBM_OK;
    for (int k = 0; k < count && rc == SLLBM_OK; ++k) {
        const int slot = k % 3;
        cudaEvent_t copied_in = ctx->pipe_ev[3 * slot], stepped = ctx->pipe_ev[3 * slot + 1],
                    copied_out = ctx->pipe_ev[3 * slot + 2];
        void* a = ctx->pipe_buf[2 * slot];
        // the slot is free once the previous state in it was copied out
        cudaError_t e = k >= 3 ? cudaStreamWaitEvent(ctx->pipe_stream[0], copied_out, 0) : cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpyAsync(a, pop_in[k], ctx->pop_bytes, cudaMemcpyHostToDevice, ctx->pipe_stream[0]);
        if (e == cudaSuccess) e = cudaEventRecord(copied_in, ctx->pipe_stream[0]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, copied_in, 0);
        if (e != cudaSuccess) {
            rc = fail(ctx, e);
            break;
        }
        ctx->buf[0] = a;
        ctx->buf[1] = ctx->pipe_buf[2 * slot + 1];
        ctx->cur = 0;
        for (int s = 0; s < n && rc == SLLBM_OK; ++s) rc = step_launch(ctx);
        if (rc != SLLBM_OK) break;
        const void* result = ctx->buf[ctx->cur];
        e = cudaEventRecord(stepped, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->pipe_stream[1], stepped, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pop_out[k], result, ctx->pop_bytes, cudaMemcpyDeviceToHost, ctx->pipe_stream[1]);
        if (e == cudaSuccess) e = cudaEventRecord(copied_out, ctx->pipe_stream[1]);
        if (e != cudaSuccess) rc = fail(ctx, e);
    }
    ctx->buf[0] = own[0];
    ctx->buf[1] = own[1];
    ctx->cur = own_cur;
    ctx->initialised = own_init;
    cudaError_t e = cudaStreamSynchronize(ctx->pipe_stream[1]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess && rc == SLLBM_OK) rc = fail(ctx, e);
    return rc;
}

int sllbm_sync(sllbm_ctx* ctx) {
    if (ctx == nullptr) return SLLBM_EINVAL;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

int sllbm_velset_d3q45(double* xi, double* w) {
    if (xi == nullptr || w == nullptr) return SLLBM_EINVAL;
    double x[kQ][3];
    double ww[kQ];
    build_velocity_set(x, ww);
    std::memcpy(xi, x, sizeof(x));
    std::memcpy(w, ww, sizeof(ww));
    return SLLBM_OK;
}

int sllbm_stream_table(int p, double h, double dt, int dir, int* shift, double* weights) {
    if (p < 2 || p > 4 || !(h > 0.0) || !(dt >= 0.0) || dir < 0 || dir > 2 || shift == nullptr
        || weights == nullptr)
        return SLLBM_EINVAL;
    double x[kQ][3];
    double ww[kQ];
    build_velocity_set(x, ww);
    DirTable* t = static_cast<DirTable*>(std::malloc(sizeof(DirTable)));
    if (t == nullptr) return SLLBM_ENOMEM;
    build_dir_table(p, h, dt, x, dir, t);
    for (int i = 0; i < kQ; ++i)
        for (int a = 0; a < p; ++a) {
            shift[i * p + a] = t->shift[i][a];
            for (int j = 0; j <= p; ++j) weights[(i * p + a) * (p + 1) + j] = t->weight[i][a][j];
        }
    std::free(t);
    return SLLBM_OK;
}

int sllbm_last_cuda_error(const sllbm_ctx* ctx) { return ctx ? ctx->last_err : 0; }

int64_t sllbm_launch_count(const sllbm_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* sllbm_strerror(int code) {
    switch (code) {
    case SLLBM_OK: return "ok";
    case SLLBM_EINVAL: return "invalid argument";
    case SLLBM_ENOMEM: return "out of memory";
    case SLLBM_ECUDA: return "CUDA runtime error";
    case SLLBM_ENONFINITE: return "non-finite or non-positive density/temperature";
    case SLLBM_ETIMEOUT: return "bounded device wait timed out";
    case SLLBM_ENOTREADY: return "populations not initialised";
    case SLLBM_EABORTED: return "step abandoned on an abort request";
    case SLLBM_EIO: return "file input/output failed";
    }
    return "unknown error";
}

}  // extern "C"
