// Fused SLLBM time step: pull streaming of the 90 populations by separable Lagrange
// interpolation + moments + equilibrium + BGK (+ Prandtl term), one tile per CTA.
//
// Data flow per CTA (tile of CX x CY x CZ cells = TX x TY x TZ nodes):
//   * each warp owns whole populations q (f_i or g_i); for one q it gathers the source
//     box of the tile (the tile translated by the velocity's departure cell shift, plus
//     one cell where the shift differs between local nodes, plus the shared face) from
//     global memory into shared memory, with periodic wrap;
//   * three separable passes (z, then y, then x) apply the per-velocity Lagrange
//     weights (Eq. interpolation; identical for every cell on the uniform mesh) and
//     leave the streamed value of every tile node in the CTA's OUT[90][tile] array;
//   * after a CTA barrier each thread takes nodes of the tile, forms rho, u, T
//     (Eq. moments), tau (Sec. II.A, Sutherland law of Sec. III.C), the fourth-order
//     equilibrium (Eq. discreteEquilibrium), and writes the collided f and g
//     (Eq. LBM, App. D) to the destination buffer.
#pragma once

#include <cstdlib>

#include "collide.cuh"
#include "sllbm_internal.h"
#include "storage.cuh"

namespace sllbm {

template <int CX, int CY, int CZ, int P>
struct TileShape {
    static constexpr int TX = CX * P, TY = CY * P, TZ = CZ * P;
    static constexpr int TILE = TX * TY * TZ;
    static constexpr int BX = (CX + 1) * P + 1, BY = (CY + 1) * P + 1, BZ = (CZ + 1) * P + 1;
    static constexpr int BOX = BX * BY * BZ;   // largest source box
    static constexpr int TMP1 = TZ * BY * BX;  // z-pass result
};

template <typename C, int P, int CX, int CY, int CZ, int NW>
struct StepSmem {
    using TS = TileShape<CX, CY, CZ, P>;
    static constexpr size_t out_elems = size_t(2) * kQ * TS::TILE;
    static constexpr size_t warp_elems = size_t(TS::BOX) + TS::TMP1;
    static constexpr size_t warp_ints = TS::BX + TS::BY + TS::BZ;
    static constexpr size_t bytes = (out_elems + NW * warp_elems) * sizeof(C) + NW * warp_ints * sizeof(int);
};

// A stored value in the arithmetic type (16-bit storage goes through FP32).
template <typename C, typename S>
__device__ __forceinline__ C load_as(S v) {
    if constexpr (PopCodec<S>::kDev)
        return static_cast<C>(static_cast<float>(v));
    else
        return static_cast<C>(v);
}

__device__ __forceinline__ int wrap_index(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Moments, equilibrium and collision of one node in 16-bit deviation storage: h[q*stride]
// holds the streamed deviations d_i = f_i/w_i - rho0 (q < 45) and d_gi = g_i/w_i - (2C_v-D)T0
// rho0 (q >= 45).  rho - rho0, rho u and 2 C_v rho (T - T0) come from deviation sums with the
// exact quadrature identities sum w = 1, sum w xi = 0, sum w |xi|^2 = D, and the collision is
// written for the deviations, so that no step subtracts quantities of the reference size:
//   d_i'  = d_i  + omega (rho (P_i - 1) + (rho - rho0) - d_i),
//   d_gi' = d_gi + omega ((2C_v-D) (T rho (P_i - 1) + (T - T0) rho + T0 (rho - rho0)) - d_gi),
// with f_i^eq = w_i rho P_i (Eq. discreteEquilibrium, P_i the quartic in xi_i.u).
template <typename S, typename C, int P, bool PR>
__device__ __forceinline__ void collide_node_dev(const C* __restrict__ h, int stride, const StepArgs& a,
                                                 const StepTables<C, P>& t, S* __restrict__ dst) {
    C drho = 0, mx = 0, my = 0, mz = 0, se = 0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const C w = t.w[i];
        const C wd = w * h[i * stride];
        drho += wd;
        mx += wd * t.xi[i][0];
        my += wd * t.xi[i][1];
        mz += wd * t.xi[i][2];
        se += wd * C(shell_xi2(shell_of(i))) + w * h[(kQ + i) * stride];
    }
    const C rho0 = C(a.rho0), T0 = C(a.T0);
    const C rho = rho0 + drho;
    const C inv_rho = C(1) / rho;
    const C ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
    const C usq = ux * ux + uy * uy + uz * uz;
    const C two_cv = C(1.0 / a.inv_2cv);
    // 2 C_v rho (T - T0) = sum w (|xi|^2 d + d_g) + D rho0 (1 - T0) - rho |u|^2 - 2 C_v T0 (rho - rho0)
    const C dT = (se + C(3) * rho0 * (C(1) - T0) - rho * usq - two_cv * T0 * drho) * inv_rho / two_cv;
    const C T = T0 + dT;
    if (a.flag != nullptr && !(rho > C(0) && T > C(0) && isfinite(rho) && isfinite(T))) atomicOr(a.flag, 1);
    const long long nn = a.nn;
    if (!a.collide) {
#pragma unroll 9
        for (int q = 0; q < 2 * kQ; ++q) dst[2 * (q % kQ) * nn + q / kQ] = static_cast<S>(static_cast<float>(h[q * stride]));
        return;
    }
    const C tau = C(a.mu_over_dt) * sutherland(T) / (rho * T) + C(0.5);
    const C om = C(1) / tau;
    const C gfac = C(a.gfac);
    const EqCoef<C> ec = eq_coefficients(usq, T - C(1));
    // App. D term from the reconstructed f_i = w_i (d_i + rho0), as in collide_node
    C Qxxx = 0, Qyyy = 0, Qzzz = 0, Qxxy = 0, Qxxz = 0, Qyyx = 0, Qyyz = 0, Qzzx = 0, Qzzy = 0,
      Qxyz = 0, ompr = 0;
    if (PR) {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const C f = t.w[i] * (h[i * stride] + rho0);
            const C cx = t.xi[i][0] - ux, cy = t.xi[i][1] - uy, cz = t.xi[i][2] - uz;
            const C fx = f * cx, fy = f * cy, fz = f * cz;
            Qxxx += fx * cx * cx;
            Qyyy += fy * cy * cy;
            Qzzz += fz * cz * cz;
            Qxxy += fx * cx * cy;
            Qxxz += fx * cx * cz;
            Qyyx += fy * cy * cx;
            Qyyz += fy * cy * cz;
            Qzzx += fz * cz * cx;
            Qzzy += fz * cz * cy;
            Qxyz += fx * cy * cz;
        }
        const C tau_pr = (tau - C(0.5)) * C(a.inv_pr) + C(0.5);
        ompr = om - C(1) / tau_pr;
    }
    const C qx = Qxxx + Qyyx + Qzzx, qy = Qxxy + Qyyy + Qzzy, qz = Qxxz + Qyyz + Qzzz;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const C x = t.xi[i][0], y = t.xi[i][1], z = t.xi[i][2];
        const C pm1 = eq_poly(ec, shell_of(i), x * ux + y * uy + z * uz) - C(1);
        const C d = h[i * stride];
        const C dg = h[(kQ + i) * stride];
        C fo = d + om * (rho * pm1 + drho - d);
        C go = dg + om * (gfac * (T * rho * pm1 + dT * rho + T0 * drho) - dg);
        if (PR) {
            const C cub = Qxxx * x * x * x + Qyyy * y * y * y + Qzzz * z * z * z
                        + C(3) * (Qxxy * x * x * y + Qxxz * x * x * z + Qyyx * y * y * x
                                  + Qyyz * y * y * z + Qzzx * z * z * x + Qzzy * z * z * y)
                        + C(6) * Qxyz * x * y * z;
            const C fst_w = C(1.0 / 6.0) * (cub - C(3) * (x * qx + y * qy + z * qz));  // f*_i / w_i
            fo += ompr * fst_w;
            go += ompr * gfac * T * fst_w;
        }
        dst[2 * i * nn] = static_cast<S>(static_cast<float>(fo));
        dst[2 * i * nn + 1] = static_cast<S>(static_cast<float>(go));
    }
}

// Moments, equilibrium and collision of one node whose streamed populations are
// h[q*stride], q = 0..89 (f then g); the result f_i, g_i goes to dst[2*i*nn + {0,1}].
template <typename S, typename C, int P, bool PR>
__device__ __forceinline__ void collide_node(const C* __restrict__ h, int stride, const StepArgs& a,
                                             const StepTables<C, P>& t, S* __restrict__ dst) {
    if constexpr (PopCodec<S>::kDev) {
        collide_node_dev<S, C, P, PR>(h, stride, a, t, dst);
        return;
    }
    C rho = 0, mx = 0, my = 0, mz = 0, e2 = 0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const C f = h[i * stride];
        rho += f;
        mx += f * t.xi[i][0];
        my += f * t.xi[i][1];
        mz += f * t.xi[i][2];
        e2 += f * C(shell_xi2(shell_of(i))) + h[(kQ + i) * stride];
    }
    const C inv_rho = C(1) / rho;
    const C ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
    const C usq = ux * ux + uy * uy + uz * uz;
    const C T = (e2 * inv_rho - usq) * C(a.inv_2cv);
    if (a.flag != nullptr && !(rho > C(0) && T > C(0) && isfinite(rho) && isfinite(T)))
        atomicOr(a.flag, 1);
    const long long nn = a.nn;
    if (!a.collide) {
#pragma unroll 9
        for (int q = 0; q < 2 * kQ; ++q)
            dst[2 * (q % kQ) * nn + q / kQ] = static_cast<S>(h[q * stride]);
        return;
    }
    // tau = mu/(P dt) + 1/2, P = rho T, mu = Sutherland(T) mu_inf  (Sec. II.A, III.C)
    const C tau = C(a.mu_over_dt) * sutherland(T) / (rho * T) + C(0.5);
    const C om = C(1) / tau;
    const C gT = C(a.gfac) * T;  // g^eq = (2 C_v - D) T f^eq
    const EqCoef<C> ec = eq_coefficients(usq, T - C(1));

    // App. D: centred third moment Qbar of the streamed f (its equilibrium part is zero
    // for this equilibrium), f*_i = (w_i/3!) Qbar : H^(3)(xi_i), g*_i = (2C_v - D) T f*_i.
    C Qxxx = 0, Qyyy = 0, Qzzz = 0, Qxxy = 0, Qxxz = 0, Qyyx = 0, Qyyz = 0, Qzzx = 0, Qzzy = 0,
      Qxyz = 0, ompr = 0;
    if (PR) {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const C f = h[i * stride];
            const C cx = t.xi[i][0] - ux, cy = t.xi[i][1] - uy, cz = t.xi[i][2] - uz;
            const C fx = f * cx, fy = f * cy, fz = f * cz;
            Qxxx += fx * cx * cx;
            Qyyy += fy * cy * cy;
            Qzzz += fz * cz * cz;
            Qxxy += fx * cx * cy;
            Qxxz += fx * cx * cz;
            Qyyx += fy * cy * cx;
            Qyyz += fy * cy * cz;
            Qzzx += fz * cz * cx;
            Qzzy += fz * cz * cy;
            Qxyz += fx * cy * cz;
        }
        const C tau_pr = (tau - C(0.5)) * C(a.inv_pr) + C(0.5);
        ompr = om - C(1) / tau_pr;
    }
    // contracted third moment q_a = sum_b Qbar_abb
    const C qx = Qxxx + Qyyx + Qzzx, qy = Qxxy + Qyyy + Qzzy, qz = Qxxz + Qyyz + Qzzz;

#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const C x = t.xi[i][0], y = t.xi[i][1], z = t.xi[i][2];
        const C s = x * ux + y * uy + z * uz;
        const C feq = t.w[i] * rho * eq_poly(ec, shell_of(i), s);
        const C f = h[i * stride];
        const C g = h[(kQ + i) * stride];
        C fo = f + om * (feq - f);
        C go = g + om * (gT * feq - g);
        if (PR) {
            // Qbar : xi xi xi over all 27 index combinations, minus 3 xi.q
            const C cub = Qxxx * x * x * x + Qyyy * y * y * y + Qzzz * z * z * z
                        + C(3) * (Qxxy * x * x * y + Qxxz * x * x * z + Qyyx * y * y * x
                                  + Qyyz * y * y * z + Qzzx * z * z * x + Qzzy * z * z * y)
                        + C(6) * Qxyz * x * y * z;
            const C fst = t.w[i] * C(1.0 / 6.0) * (cub - C(3) * (x * qx + y * qy + z * qz));
            fo += ompr * fst;
            go += ompr * gT * fst;
        }
        dst[2 * i * nn] = static_cast<S>(fo);
        dst[2 * i * nn + 1] = static_cast<S>(go);
    }
}

template <typename S, typename C, int P, int CX, int CY, int CZ, int NW, bool PR>
__global__ void __launch_bounds__(NW * 32, 1)
    step_kernel(const StepArgs a, const __grid_constant__ StepTables<C, P> t) {
    using TS = TileShape<CX, CY, CZ, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* out = reinterpret_cast<C*>(smem_raw);
    C* wbase = out + StepSmem<C, P, CX, CY, CZ, NW>::out_elems;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* box = wbase + warp * (TS::BOX + TS::TMP1);
    C* tmp1 = box + TS::BOX;
    int* xo = reinterpret_cast<int*>(wbase + NW * (TS::BOX + TS::TMP1)) + warp * (TS::BX + TS::BY + TS::BZ);
    int* yo = xo + TS::BX;
    int* zo = yo + TS::BY;

    int tile = blockIdx.x;
    const int tix = tile % a.tiles[0];
    tile /= a.tiles[0];
    const int tiy = tile % a.tiles[1];
    const int tiz = tile / a.tiles[1];
    const int c0[3] = {tix * CX, tiy * CY, tiz * CZ};
    const int tc[3] = {min(CX, a.cells[0] - c0[0]), min(CY, a.cells[1] - c0[1]), min(CZ, a.cells[2] - c0[2])};
    const int te[3] = {tc[0] * P, tc[1] * P, tc[2] * P};
    const S* __restrict__ src = static_cast<const S*>(a.src);
    const int nxy = a.N[0] * a.N[1];

    for (int q = warp; q < 2 * kQ; q += NW) {
        const int i = q < kQ ? q : q - kQ;
        int s[3], b0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s[d] = (tc[d] + t.span[i][d]) * P + 1;
            b0[d] = (c0[d] + t.kmin[i][d]) * P;
        }
        for (int e = lane; e < s[0]; e += 32) xo[e] = wrap_index(b0[0] + e, a.N[0]);
        for (int e = lane; e < s[1]; e += 32) yo[e] = wrap_index(b0[1] + e, a.N[1]) * a.N[0];
        for (int e = lane; e < s[2]; e += 32) zo[e] = wrap_index(b0[2] + e, a.N[2]) * nxy;
        __syncwarp();
        // storage order [i][node][h]: population q = (h, i) is every second element
        const S* __restrict__ sq = src + 2LL * i * a.nn + (q < kQ ? 0 : 1);
        const int sxy = s[0] * s[1];
        const int tot = sxy * s[2];
        for (int e = lane; e < tot; e += 32) {
            const int z = e / sxy;
            const int r = e - z * sxy;
            const int y = r / s[0];
            const int x = r - y * s[0];
            box[e] = load_as<C>(__ldg(sq + 2 * (zo[z] + yo[y] + xo[x])));
        }
        __syncwarp();
        // z pass: tmp1[oz][y][x] = sum_l Lz[az][l] box[zb+l][y][x]
        const int n1 = te[2] * sxy;
        for (int e = lane; e < n1; e += 32) {
            const int oz = e / sxy;
            const int r = e - oz * sxy;
            const int az = oz % P;
            const int zb = (oz / P + t.kc[i][2][az]) * P;
            C acc = 0;
#pragma unroll
            for (int l = 0; l <= P; ++l) acc += t.lw[i][2][az][l] * box[(zb + l) * sxy + r];
            tmp1[e] = acc;
        }
        __syncwarp();
        // y pass: box[oz][oy][x] = sum_k Ly[ay][k] tmp1[oz][yb+k][x]
        const int n2 = te[2] * te[1] * s[0];
        for (int e = lane; e < n2; e += 32) {
            const int x = e % s[0];
            const int r = e / s[0];
            const int oy = r % te[1];
            const int oz = r / te[1];
            const int ay = oy % P;
            const int yb = (oy / P + t.kc[i][1][ay]) * P;
            C acc = 0;
#pragma unroll
            for (int k = 0; k <= P; ++k) acc += t.lw[i][1][ay][k] * tmp1[(oz * s[1] + yb + k) * s[0] + x];
            box[e] = acc;
        }
        __syncwarp();
        // x pass: OUT[q][oz][oy][ox] = sum_j Lx[ax][j] box[oz][oy][xb+j]
        const int n3 = te[2] * te[1] * te[0];
        C* oq = out + q * TS::TILE;
        for (int e = lane; e < n3; e += 32) {
            const int ox = e % te[0];
            const int r = e / te[0];
            const int oy = r % te[1];
            const int oz = r / te[1];
            const int ax = ox % P;
            const int xb = (ox / P + t.kc[i][0][ax]) * P;
            C acc = 0;
#pragma unroll
            for (int j = 0; j <= P; ++j) acc += t.lw[i][0][ax][j] * box[(oz * te[1] + oy) * s[0] + xb + j];
            oq[(oz * TS::TY + oy) * TS::TX + ox] = acc;
        }
        __syncwarp();
    }
    __syncthreads();

    S* dst = static_cast<S*>(a.dst);
    for (int n = threadIdx.x; n < TS::TILE; n += NW * 32) {
        const int ox = n % TS::TX;
        const int r = n / TS::TX;
        const int oy = r % TS::TY;
        const int oz = r / TS::TY;
        if (ox >= te[0] || oy >= te[1] || oz >= te[2]) continue;
        const long long g = (static_cast<long long>(c0[2] * P + oz) * a.N[1] + (c0[1] * P + oy)) * a.N[0]
                          + (c0[0] * P + ox);
        collide_node<S, C, P, PR>(out + n, TS::TILE, a, t, dst + 2 * g);
    }
}

// WITH_PR = false instantiates only the kernel without the Prandtl term (tile-shape
// variants offered to the autotuner); such a launcher refuses contexts with the term on.
template <typename S, typename C, int P, int CX, int CY, int CZ, int NW, bool WITH_PR = true>
int launch_step_tiled(sllbm_ctx* ctx, const void* src, void* dst) {
    if (!WITH_PR && ctx->prm.pr_correction) return SLLBM_EINVAL;
    using SM = StepSmem<C, P, CX, CY, CZ, NW>;
    static_assert(SM::bytes <= 227 * 1024, "shared memory budget");
    // the tables are built once per context and kept in its host-side blob
    if (ctx->step_blob == nullptr || ctx->step_blob_size != sizeof(StepTables<C, P>)) {
        free(ctx->step_blob);
        ctx->step_blob = static_cast<unsigned char*>(malloc(sizeof(StepTables<C, P>)));
        if (ctx->step_blob == nullptr) return SLLBM_ENOMEM;
        ctx->step_blob_size = sizeof(StepTables<C, P>);
        fill_step_tables<C, P>(ctx, reinterpret_cast<StepTables<C, P>*>(ctx->step_blob));
    }
    const StepTables<C, P>* tab = reinterpret_cast<const StepTables<C, P>*>(ctx->step_blob);
    StepArgs args;
    fill_step_args(ctx, src, dst, &args);
    args.tiles[0] = (ctx->cells[0] + CX - 1) / CX;
    args.tiles[1] = (ctx->cells[1] + CY - 1) / CY;
    args.tiles[2] = (ctx->cells[2] + CZ - 1) / CZ;
    const long long ntiles = static_cast<long long>(args.tiles[0]) * args.tiles[1] * args.tiles[2];
    if (ntiles > 0x7fffffffLL) return SLLBM_EINVAL;
    cudaError_t err = cudaSuccess;
    if (ctx->prm.pr_correction) {
        if constexpr (WITH_PR) {
            auto k = step_kernel<S, C, P, CX, CY, CZ, NW, true>;
            err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SM::bytes));
            if (err == cudaSuccess) {
                k<<<static_cast<unsigned>(ntiles), NW * 32, SM::bytes, ctx->stream>>>(args, *tab);
                err = cudaGetLastError();
            }
        }
    } else {
        auto k = step_kernel<S, C, P, CX, CY, CZ, NW, false>;
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SM::bytes));
        if (err == cudaSuccess) {
            k<<<static_cast<unsigned>(ntiles), NW * 32, SM::bytes, ctx->stream>>>(args, *tab);
            err = cudaGetLastError();
        }
    }
    ctx->launches += 1;
    if (err != cudaSuccess) {
        ctx->last_err = static_cast<int>(err);
        return SLLBM_ECUDA;
    }
    return SLLBM_OK;
}

}  // namespace sllbm
