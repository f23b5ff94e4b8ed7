// Fused SLLBM time step: pull streaming of the 90 populations by separable Lagrange
// interpolation + moments + equilibrium + BGK (+ Prandtl term), one tile per CTA.
//
// Data flow per CTA (tile of CX x CY x CZ cells = TX x TY x TZ nodes):
//   * each warp owns whole velocity pairs (f_i, g_i), which share departure points and
//     weights; for one pair, each lane takes columns (x, y) of the pair's source box (the
//     tile translated by the velocity's departure cell shift, plus one cell where the shift
//     differs between local nodes, plus the shared face), loads the column's values from
//     global memory into registers (periodic wrap, all loads of a column issued together)
//     and applies the z pass there (Eq. interpolation; the weights are identical for every
//     cell on the uniform mesh), writing the TZ output planes to a per-warp buffer;
//   * the y pass runs in place over columns (x, z) of that buffer, the x pass over rows
//     (y, z), leaving the streamed f_i and g_i of every tile node in the CTA's OUT[90][tile];
//     which of two candidate support ranges a local node uses is a register select, not a
//     computed register index;
//   * after a CTA barrier each thread takes nodes of the tile, forms rho, u, T
//     (Eq. moments), tau (Sec. II.A, Sutherland law of Sec. III.C), the fourth-order
//     equilibrium (Eq. discreteEquilibrium), and writes the collided f and g
//     (Eq. LBM, App. D) to the destination buffer.
#pragma once

#include <cstdlib>
#include <type_traits>

#include "collide.cuh"
#include "compsum.cuh"
#include "packed.cuh"
#include "sllbm_internal.h"
#include "storage.cuh"

namespace sllbm {

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

template <int CX, int CY, int CZ, int P>
struct TileShape {
    static constexpr int TX = CX * P, TY = CY * P, TZ = CZ * P;
    static constexpr int TILE = TX * TY * TZ;
    static constexpr int BX = (CX + 1) * P + 1, BY = (CY + 1) * P + 1, BZ = (CZ + 1) * P + 1;
    // OUT holds the streamed value of node (row r = oz TY + oy, ox) at r TX + (ox + r / RG) % TX,
    // RG = 32 / gcd(TX W, 32) for values of W 4-byte words: rows RG apart start on the same
    // bank, so each group of RG rows is rotated by one more place, and the x pass's stores
    // (one row per lane) fall on distinct banks
    template <int W>
    static constexpr int RG = 32 / gcd_c(TX * W, 32);
    template <int W>
    __host__ __device__ static constexpr int slot(int r, int ox) {
        return r * TX + (ox + r / RG<W>) % TX;
    }
};

// Pair of the arithmetic type (f_i, g_i).
template <typename C>
struct Pair2;
template <>
struct Pair2<float> {
    using T = float2;
};
template <>
struct Pair2<double> {
    using T = double2;
};

template <typename C, int P, int CX, int CY, int CZ, int NW>
struct StepSmem {
    using TS = TileShape<CX, CY, CZ, P>;
    using C2 = typename Pair2<C>::T;
    static constexpr size_t out_elems = size_t(2) * kQ * TS::TILE;
    static constexpr size_t out_bytes = (out_elems * sizeof(C) + 15) / 16 * 16;
    // z-pass output planes; rows padded to an odd number of pairs (see step_tile)
    static constexpr size_t warp_pairs = size_t(TS::TZ) * TS::BY * (TS::BX | 1);
    static constexpr size_t warp_ints = TS::BX + TS::BY + TS::BZ;
    static constexpr size_t bytes = out_bytes + NW * warp_pairs * sizeof(C2) + NW * warp_ints * sizeof(int);
};

// One stored pair (f_i, g_i) widened to the arithmetic type.
template <typename C, typename S>
__device__ __forceinline__ typename Pair2<C>::T load_pair(const S* p) {
    typename Pair2<C>::T r;
    if constexpr (std::is_same<S, float>::value) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        r.x = static_cast<C>(v.x);
        r.y = static_cast<C>(v.y);
    } else if constexpr (std::is_same<S, double>::value) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        r.x = static_cast<C>(v.x);
        r.y = static_cast<C>(v.y);
    } else if constexpr (std::is_same<S, __half>::value) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
        r.x = static_cast<C>(v.x);
        r.y = static_cast<C>(v.y);
    } else {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        r.x = static_cast<C>(v.x);
        r.y = static_cast<C>(v.y);
    }
    return r;
}

template <typename C, int P>
__device__ __forceinline__ void load_pass_weights(const C (&w)[P][P + 1], const signed char (&kc)[P],
                                                  C (&wr)[P][P + 1], signed char (&kr)[P]) {
#pragma unroll
    for (int a = 0; a < P; ++a) {
        kr[a] = kc[a];
#pragma unroll
        for (int l = 0; l <= P; ++l) wr[a][l] = w[a][l];
    }
}

// One 1D Lagrange pass over a column held in registers: output o (0..T-1, local index
// a = o % P in cell o / P) = sum_l w[a][l] v[(o/P + k_a) P + l] with k_a in {0, 1}.
template <typename C, int P, int T, int NV>
__device__ __forceinline__ void lagrange_column(const typename Pair2<C>::T (&v)[NV], const C (&w)[P][P + 1],
                                                const signed char (&kc)[P], typename Pair2<C>::T (&r)[T]) {
#pragma unroll
    for (int o = 0; o < T; ++o) {
        const int a = o % P;
        const int base = (o / P) * P;
        const bool hi = kc[a] != 0;
        C fx = 0, fy = 0;
#pragma unroll
        for (int l = 0; l <= P; ++l) {
            const C wl = w[a][l];
            const int lo_i = base + l, hi_i = base + P + l;
            static_assert((T - 1) / P * P + 2 * P < NV, "column shorter than the support of its outputs");
            const C vx = hi ? v[hi_i].x : v[lo_i].x;
            const C vy = hi ? v[hi_i].y : v[lo_i].y;
            fx += wl * vx;
            fy += wl * vy;
        }
        r[o].x = fx;
        r[o].y = fy;
    }
}

// FP32 form of a pass without selects: for local node a the 2P+1 taps over v[base .. base+2P]
// carry the P+1 weights at offset k_a P and zeros elsewhere, each as the pair (w, w) for the
// packed FMA.  The real taps keep their order and a zero tap adds exactly zero, so a column
// gives the same values as lagrange_column.
template <int P>
__device__ __forceinline__ void pad_weights(const float (&w)[P][P + 1], const signed char (&kc)[P],
                                            float2 (&W)[P][2 * P + 1]) {
#pragma unroll
    for (int a = 0; a < P; ++a) {
#pragma unroll
        for (int m = 0; m <= 2 * P; ++m) {
            const float lo = m <= P ? w[a][m] : 0.f;
            const float hi = m >= P ? w[a][m - P] : 0.f;
            const float x = kc[a] != 0 ? hi : lo;
            W[a][m] = make_float2(x, x);
        }
    }
}

template <int P, int T, int NV>
__device__ __forceinline__ void lagrange_column_packed(const float2 (&v)[NV], const float2 (&W)[P][2 * P + 1],
                                                       float2 (&r)[T]) {
    static_assert((T - 1) / P * P + 2 * P < NV, "column shorter than the taps of its outputs");
#pragma unroll
    for (int o = 0; o < T; ++o) {
        const int a = o % P;
        const int base = (o / P) * P;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m <= 2 * P; ++m) acc = ffma2(v[base + m], W[a][m], acc);
        r[o] = acc;
    }
}

// The weights of one pass of one velocity pair, held in registers for its columns, and the
// pass over a column: register selects for FP64 arithmetic (padding would add FP64 FMAs),
// the packed select-free form for FP32 arithmetic.
template <typename C, int P>
struct ColumnPass {
    C w[P][P + 1];
    signed char k[P];
    __device__ __forceinline__ void load(const C (&lw)[P][P + 1], const signed char (&kc)[P]) {
        load_pass_weights<C, P>(lw, kc, w, k);
    }
    template <int T, int NV>
    __device__ __forceinline__ void apply(const typename Pair2<C>::T (&v)[NV], typename Pair2<C>::T (&r)[T]) const {
        lagrange_column<C, P, T, NV>(v, w, k, r);
    }
};

template <int P>
struct ColumnPass<float, P> {
    float2 W[P][2 * P + 1];
    __device__ __forceinline__ void load(const float (&lw)[P][P + 1], const signed char (&kc)[P]) {
        float w[P][P + 1];
        signed char k[P];
        load_pass_weights<float, P>(lw, kc, w, k);
        pad_weights<P>(w, k, W);
    }
    template <int T, int NV>
    __device__ __forceinline__ void apply(const float2 (&v)[NV], float2 (&r)[T]) const {
        lagrange_column_packed<P, T, NV>(v, W, r);
    }
};

// One pair (f_i, g_i) stored with a single 2-element store (the pair is adjacent in a state
// buffer and aligned to its size).
template <typename S, typename C>
__device__ __forceinline__ void store_pair(S* p, C f, C g) {
    if constexpr (std::is_same<S, float>::value) {
        *reinterpret_cast<float2*>(p) = make_float2(static_cast<float>(f), static_cast<float>(g));
    } else if constexpr (std::is_same<S, double>::value) {
        *reinterpret_cast<double2*>(p) = make_double2(static_cast<double>(f), static_cast<double>(g));
    } else if constexpr (std::is_same<S, __half>::value) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(static_cast<float>(f), static_cast<float>(g));
    } else {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(static_cast<float>(f), static_cast<float>(g));
    }
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
template <typename S, typename C, int P, bool PR, class LT, bool KC = false>
__device__ __forceinline__ void collide_node_dev(const C* __restrict__ h, int stride, const StepArgs& a,
                                                 const LT& t, S* __restrict__ dst) {
    C drho = 0, mx = 0, my = 0, mz = 0, se = 0;
    const C rho0 = C(a.rho0), T0 = C(a.T0);
    const C two_cv = C(1.0 / a.inv_2cv);
    C rho, inv_rho, ux, uy, uz, usq, dT;
    if constexpr (KC) {
        // compensated sums of the deviation moments, and of the energy balance below
        CompSum<C> r, qx, qy, qz, e;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const C w = t.w[i];
            const C d = h[i * stride];
            r.add_prod(w, d);
            qx.add_prod(w * t.xi[i][0], d);
            qy.add_prod(w * t.xi[i][1], d);
            qz.add_prod(w * t.xi[i][2], d);
            e.add_prod(w * C(shell_xi2(shell_of(i))), d);
            e.add_prod(w, h[(kQ + i) * stride]);
        }
        drho = r.value();
        mx = qx.value();
        my = qy.value();
        mz = qz.value();
        rho = rho0 + drho;
        inv_rho = C(1) / rho;
        ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
        usq = ux * ux + uy * uy + uz * uz;
        // 2 C_v rho (T - T0) with rho |u|^2 = m . u and every term compensated
        e.add(C(3) * rho0 * (C(1) - T0));
        e.add_prod(-mx, ux);
        e.add_prod(-my, uy);
        e.add_prod(-mz, uz);
        e.add_prod(-two_cv * T0, drho);
        dT = e.value() * inv_rho / two_cv;
    } else {
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
        rho = rho0 + drho;
        inv_rho = C(1) / rho;
        ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
        usq = ux * ux + uy * uy + uz * uz;
        // 2 C_v rho (T - T0) = sum w (|xi|^2 d + d_g) + D rho0 (1 - T0) - rho |u|^2 - 2 C_v T0 (rho - rho0)
        dT = (se + C(3) * rho0 * (C(1) - T0) - rho * usq - two_cv * T0 * drho) * inv_rho / two_cv;
    }
    const C T = T0 + dT;
    if (a.flag != nullptr && !(rho > C(0) && T > C(0) && isfinite(rho) && isfinite(T))) atomicOr(a.flag, 1);
    const long long nn = a.nn;
    if (!a.collide) {
#pragma unroll 9
        for (int i = 0; i < kQ; ++i) store_pair<S>(dst + 2 * i * nn, h[i * stride], h[(kQ + i) * stride]);
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
        store_pair<S>(dst + 2 * i * nn, fo, go);
    }
}

// Moments, equilibrium and collision of one node whose streamed populations are
// h[q*stride], q = 0..89 (f then g); the result f_i, g_i goes to dst[2*i*nn + {0,1}].  The
// velocity set comes from t.xi, t.w (a StepTables or a Lattice).
template <typename S, typename C, int P, bool PR, class LT, bool KC = false>
__device__ __forceinline__ void collide_node(const C* __restrict__ h, int stride, const StepArgs& a,
                                             const LT& t, S* __restrict__ dst) {
    if constexpr (PopCodec<S>::kDev) {
        collide_node_dev<S, C, P, PR, LT, KC>(h, stride, a, t, dst);
        return;
    }
    const long long nn = a.nn;
    if (!a.collide) {  // streaming only: store the streamed pairs
#pragma unroll 9
        for (int i = 0; i < kQ; ++i) store_pair<S>(dst + 2 * i * nn, h[i * stride], h[(kQ + i) * stride]);
        return;
    }
    C rho = 0, mx = 0, my = 0, mz = 0, e2 = 0;
    C inv_rho, ux, uy, uz, usq, T;
    if constexpr (KC) {
        // compensated moment sums, and 2 rho E - rho |u|^2 = 2 rho E - m . u compensated
        CompSum<C> r, qx, qy, qz, e;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const C f = h[i * stride];
            r.add(f);
            qx.add_prod(f, t.xi[i][0]);
            qy.add_prod(f, t.xi[i][1]);
            qz.add_prod(f, t.xi[i][2]);
            e.add_prod(f, C(shell_xi2(shell_of(i))));
            e.add(h[(kQ + i) * stride]);
        }
        rho = r.value();
        mx = qx.value();
        my = qy.value();
        mz = qz.value();
        inv_rho = C(1) / rho;
        ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
        usq = ux * ux + uy * uy + uz * uz;
        e.add_prod(-mx, ux);
        e.add_prod(-my, uy);
        e.add_prod(-mz, uz);
        T = e.value() * inv_rho * C(a.inv_2cv);
    } else {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const C f = h[i * stride];
            rho += f;
            mx += f * t.xi[i][0];
            my += f * t.xi[i][1];
            mz += f * t.xi[i][2];
            e2 += f * C(shell_xi2(shell_of(i))) + h[(kQ + i) * stride];
        }
        inv_rho = C(1) / rho;
        ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
        usq = ux * ux + uy * uy + uz * uz;
        T = (e2 * inv_rho - usq) * C(a.inv_2cv);
    }
    if (a.flag != nullptr && !(rho > C(0) && T > C(0) && isfinite(rho) && isfinite(T)))
        atomicOr(a.flag, 1);
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
        store_pair<S>(dst + 2 * i * nn, fo, go);
    }
}

// First velocity of shell sh in the canonical order (0, 1, 13, 33; 45 past the last).
__host__ __device__ constexpr int shell_begin(int sh) {
    return sh <= 0 ? 0 : (sh == 1 ? 1 : (sh == 2 ? 13 : (sh == 3 ? 33 : 45)));
}

// collide_node for two lanes (lane pair 2k, 2k+1, `mask` naming both) sharing one node: the
// lane with parity `half` takes the velocities i with i % 2 == half, shell by shell (the
// shell's equilibrium coefficients stay compile-time indexed); the moment sums are combined
// with one exchange, and both lanes form the node's parameters.  Storage types that hold the
// populations themselves, no Prandtl term.
template <typename S, typename C, int P, class LT>
__device__ __forceinline__ void collide_node_pair(const C* __restrict__ h, int stride, const StepArgs& a,
                                                  const LT& t, S* __restrict__ dst, int half,
                                                  unsigned mask) {
    if (!a.collide) {  // streaming only: each lane stores its velocities' pairs
        for (int i = half; i < kQ; i += 2) store_pair<S>(dst + 2 * i * a.nn, h[i * stride], h[(kQ + i) * stride]);
        return;
    }
    // shells 1, 2, 3 hold 12, 20, 12 velocities (6, 10, 6 per lane); the origin goes to lane 0
    constexpr int kPer[4] = {1, 6, 10, 6};
    C rho = 0, mx = 0, my = 0, mz = 0, e2 = 0;
#pragma unroll
    for (int sh = 0; sh < 4; ++sh) {
        const C x2 = C(shell_xi2(sh));
        const int i0 = shell_begin(sh) + ((shell_begin(sh) ^ half) & 1);
#pragma unroll
        for (int m = 0; m < kPer[sh]; ++m) {
            const int i = i0 + 2 * m;
            if (sh == 0 && half != 0) break;
            const C f = h[i * stride];
            rho += f;
            mx += f * t.xi[i][0];
            my += f * t.xi[i][1];
            mz += f * t.xi[i][2];
            e2 += f * x2 + h[(kQ + i) * stride];
        }
    }
    rho += __shfl_xor_sync(mask, rho, 1);
    mx += __shfl_xor_sync(mask, mx, 1);
    my += __shfl_xor_sync(mask, my, 1);
    mz += __shfl_xor_sync(mask, mz, 1);
    e2 += __shfl_xor_sync(mask, e2, 1);
    const C inv_rho = C(1) / rho;
    const C ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
    const C usq = ux * ux + uy * uy + uz * uz;
    const C T = (e2 * inv_rho - usq) * C(a.inv_2cv);
    if (half == 0 && a.flag != nullptr && !(rho > C(0) && T > C(0) && isfinite(rho) && isfinite(T)))
        atomicOr(a.flag, 1);
    const long long nn = a.nn;
    // tau = mu/(P dt) + 1/2, P = rho T, mu = Sutherland(T) mu_inf  (Sec. II.A, III.C)
    const C tau = C(a.mu_over_dt) * sutherland(T) / (rho * T) + C(0.5);
    const C om = C(1) / tau;
    const C gT = C(a.gfac) * T;  // g^eq = (2 C_v - D) T f^eq
    const EqCoef<C> ec = eq_coefficients(usq, T - C(1));
#pragma unroll
    for (int sh = 0; sh < 4; ++sh) {
        const C c0 = ec.c0[sh], c1 = ec.c1[sh], c2 = ec.c2[sh];
        const int i0 = shell_begin(sh) + ((shell_begin(sh) ^ half) & 1);
#pragma unroll
        for (int m = 0; m < kPer[sh]; ++m) {
            const int i = i0 + 2 * m;
            if (sh == 0 && half != 0) break;
            const C s = t.xi[i][0] * ux + t.xi[i][1] * uy + t.xi[i][2] * uz;
            const C feq =
                t.w[i] * rho * (c0 + s * (c1 + s * (c2 + s * (C(1.0 / 6.0) + s * C(1.0 / 24.0)))));
            const C f = h[i * stride];
            const C g = h[(kQ + i) * stride];
            store_pair<S>(dst + 2 * i * nn, f + om * (feq - f), g + om * (gT * feq - g));
        }
    }
}

// Per-node phase of the step: moments, equilibrium, collision, store (Eq. LBM).  Two lanes
// per node (kPair) are possible where the storage holds the populations themselves and the
// Prandtl term is off; step_tile uses them on tiles much smaller than the CTA.
template <typename S, typename C, int P, bool PR, bool KC = false>
struct CollideOp {
    static constexpr bool kPair = !PR && !KC && !PopCodec<S>::kDev;
    __device__ __forceinline__ void operator()(const C* h, int stride, const StepArgs& a, const StepTables<C, P>& t,
                                               long long g) const {
        collide_node<S, C, P, PR, StepTables<C, P>, KC>(h, stride, a, t, static_cast<S*>(a.dst) + 2 * g);
    }
    __device__ __forceinline__ void pair(const C* h, int stride, const StepArgs& a, const StepTables<C, P>& t,
                                         long long g, int half, unsigned mask) const {
        collide_node_pair<S, C, P>(h, stride, a, t, static_cast<S*>(a.dst) + 2 * g, half, mask);
    }
};

// CollideOp of the batched kernel: the velocity set is read from `lat` (a kernel parameter,
// shared by every mesh) instead of the job's tables, which that kernel keeps in shared
// memory; collision operands then come from the constant bank as in step_kernel.
template <typename C, int P>
struct LatticeCollideOp {
    static constexpr bool kPair = true;
    const Lattice<C>& lat;
    __device__ __forceinline__ void operator()(const C* h, int stride, const StepArgs& a, const StepTables<C, P>&,
                                               long long g) const {
        collide_node<C, C, P, false>(h, stride, a, lat, static_cast<C*>(a.dst) + 2 * g);
    }
    __device__ __forceinline__ void pair(const C* h, int stride, const StepArgs& a, const StepTables<C, P>&,
                                         long long g, int half, unsigned mask) const {
        collide_node_pair<C, C, P>(h, stride, a, lat, static_cast<C*>(a.dst) + 2 * g, half, mask);
    }
};

// The step of one tile (tile index `tile` of the mesh a describes), all NW warps of the CTA,
// with the CTA's dynamic shared memory at smem_raw: streaming of the 90 populations of the
// tile's nodes into shared memory, then op(streamed values of node n (stride TILE), a, t,
// global node index) for every node of the tile.  Used by step_kernel (one tile per CTA),
// by the batched persistent kernel (many tiles of many meshes per CTA) and, with the
// collision's vector-Jacobian product as op, by the reverse mode.
template <typename S, typename C, int P, int CX, int CY, int CZ, int NW, bool PR, class Op>
__device__ __forceinline__ void step_tile(const StepArgs& a, const StepTables<C, P>& t, int tile,
                                          unsigned char* smem_raw, Op& op) {
    using TS = TileShape<CX, CY, CZ, P>;
    using SM = StepSmem<C, P, CX, CY, CZ, NW>;
    using C2 = typename Pair2<C>::T;
    C* out = reinterpret_cast<C*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C2* zb = reinterpret_cast<C2*>(smem_raw + SM::out_bytes) + warp * SM::warp_pairs;
    int* xo = reinterpret_cast<int*>(smem_raw + SM::out_bytes + NW * SM::warp_pairs * sizeof(C2)) +
              warp * SM::warp_ints;
    int* yo = xo + TS::BX;
    int* zo = yo + TS::BY;

    const int tix = tile % a.tiles[0];
    tile /= a.tiles[0];
    const int tiy = tile % a.tiles[1];
    const int tiz = tile / a.tiles[1] + a.tz_begin;
    // (a slab's tiles cover its interior cells, which start a.z0 cells above its first plane)
    const int c0[3] = {tix * CX, tiy * CY, tiz * CZ + a.z0};
    const int tc[3] = {min(CX, a.cells[0] - c0[0]), min(CY, a.cells[1] - c0[1]),
                       min(CZ, a.cells[2] + a.z0 - c0[2])};
    const int te[3] = {tc[0] * P, tc[1] * P, tc[2] * P};
    const S* __restrict__ src = static_cast<const S*>(a.src);
    const int nxy = a.N[0] * a.N[1];

    for (int i = warp; i < kQ; i += NW) {
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
        // storage order [i][node][h]: the pair (f_i, g_i) of a node is two adjacent values
        const S* __restrict__ sp = src + 2LL * i * a.nn;
        const int sx = s[0], sxy = s[0] * s[1];
        // rows of the per-warp buffer hold an odd number of pairs, so that the x pass's lanes
        // (one row each) fall on different banks; planes are s[1] such rows
        const int rs = sx | 1, ps = rs * s[1];
        // each pass reads the pair's weights and departure-cell bits of its direction from
        // the constant bank once, before its column loop
        ColumnPass<C, P> pz;
        pz.load(t.lw[i][2], t.kc[i][2]);
        // gather + z pass: lane = column (x, y) of the source box
        for (int col = lane; col < sxy; col += 32) {
            const int y = col / sx;
            const int x = col - y * sx;
            const int off = yo[y] + xo[x];
            C2 v[TS::BZ];
#pragma unroll
            for (int z = 0; z < TS::BZ; ++z) {
                if (z < s[2]) {
                    v[z] = load_pair<C>(sp + 2LL * (zo[z] + off));
                } else {
                    v[z].x = C(0);
                    v[z].y = C(0);
                }
            }
            C2 r[TS::TZ];
            pz.template apply<TS::TZ, TS::BZ>(v, r);
#pragma unroll
            for (int oz = 0; oz < TS::TZ; ++oz)
                if (oz < te[2]) zb[oz * ps + y * rs + x] = r[oz];
        }
        __syncwarp();
        // y pass in place: lane = column (x, z)
        ColumnPass<C, P> py;
        py.load(t.lw[i][1], t.kc[i][1]);
        const int ncol = te[2] * sx;
        for (int col = lane; col < ncol; col += 32) {
            const int oz = col / sx;
            const int x = col - oz * sx;
            C2* cp = zb + oz * ps + x;
            C2 v[TS::BY];
#pragma unroll
            for (int y = 0; y < TS::BY; ++y) {
                if (y < s[1]) {
                    v[y] = cp[y * rs];
                } else {
                    v[y].x = C(0);
                    v[y].y = C(0);
                }
            }
            C2 r[TS::TY];
            py.template apply<TS::TY, TS::BY>(v, r);
#pragma unroll
            for (int oy = 0; oy < TS::TY; ++oy)
                if (oy < te[1]) cp[oy * rs] = r[oy];
        }
        __syncwarp();
        // x pass: lane = row (y, z) of the tile; f_i to OUT[i], g_i to OUT[45 + i]
        ColumnPass<C, P> px;
        px.load(t.lw[i][0], t.kc[i][0]);
        for (int row = lane; row < TS::TY * TS::TZ; row += 32) {
            const int oz = row / TS::TY;
            const int oy = row - oz * TS::TY;
            if (oz >= te[2] || oy >= te[1]) continue;
            const C2* rp = zb + oz * ps + oy * rs;
            C2 v[TS::BX];
#pragma unroll
            for (int x = 0; x < TS::BX; ++x) {
                if (x < sx) {
                    v[x] = rp[x];
                } else {
                    v[x].x = C(0);
                    v[x].y = C(0);
                }
            }
            C2 r[TS::TX];
            px.template apply<TS::TX, TS::BX>(v, r);
            C* of = out + i * TS::TILE + row * TS::TX;  // (row = oz TY + oy)
            C* og = of + kQ * TS::TILE;
            const int rot = (row / TS::template RG<int(sizeof(C) / 4)>) % TS::TX;
#pragma unroll
            for (int ox = 0; ox < TS::TX; ++ox) {
                if (ox < te[0]) {
                    const int c = ox + rot < TS::TX ? ox + rot : ox + rot - TS::TX;
                    of[c] = r[ox].x;
                    og[c] = r[ox].y;
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();

    // Two lanes per node only where the tile has at most a quarter as many nodes as the CTA
    // has threads (measured: on the larger default tiles one lane per node, with its fully
    // unrolled velocity loops, is faster).
    if constexpr (Op::kPair && 4 * TS::TILE <= NW * 32) {
        // two lanes per node: k = 2 n + half, the pair in one warp (NW * 32 is even)
        for (int k = threadIdx.x; k < 2 * TS::TILE; k += NW * 32) {
            const int n = k >> 1;
            const int ox = n % TS::TX;
            const int r = n / TS::TX;
            const int oy = r % TS::TY;
            const int oz = r / TS::TY;
            if (ox >= te[0] || oy >= te[1] || oz >= te[2]) continue;  // both lanes of the pair
            const long long g = (static_cast<long long>(c0[2] * P + oz) * a.N[1] + (c0[1] * P + oy)) * a.N[0]
                              + (c0[0] * P + ox);
            op.pair(out + TS::template slot<int(sizeof(C) / 4)>(r, ox), TS::TILE, a, t, g, k & 1, 3u << (lane & 30));
        }
    } else {
        for (int n = threadIdx.x; n < TS::TILE; n += NW * 32) {
            const int ox = n % TS::TX;
            const int r = n / TS::TX;
            const int oy = r % TS::TY;
            const int oz = r / TS::TY;
            if (ox >= te[0] || oy >= te[1] || oz >= te[2]) continue;
            const long long g = (static_cast<long long>(c0[2] * P + oz) * a.N[1] + (c0[1] * P + oy)) * a.N[0]
                              + (c0[0] * P + ox);
            op(out + TS::template slot<int(sizeof(C) / 4)>(r, ox), TS::TILE, a, t, g);
        }
    }
}

// CTAs per SM the registers are sized for: two for 9-warp tiles with FP32 arithmetic (the
// p = 3 default, whose shared memory fits twice and whose 45 velocity pairs split evenly, 5
// per warp), one otherwise.
template <typename C, int NW>
constexpr int kStepMinCtas = NW == 9 && sizeof(C) == 4 ? 2 : 1;

template <typename S, typename C, int P, int CX, int CY, int CZ, int NW, bool PR, bool KC = false>
__global__ void __launch_bounds__(NW * 32, kStepMinCtas<C, NW>)
    step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ StepTables<C, P> t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CollideOp<S, C, P, PR, KC> op;
    step_tile<S, C, P, CX, CY, CZ, NW, PR>(a, t, blockIdx.x, smem_raw, op);
}

// Many meshes of one order in one launch: job k of the list (BatchJob) owns work items
// [tile_begin_k, tile_begin_{k+1}) (its tiles in order); persistent CTAs walk the items with
// a grid stride.
// Shared memory of the batched kernel: the tile body's, then the current job's tables and
// arguments (copied from global memory when a CTA moves to another job).
template <typename C, int P, int CX, int CY, int CZ, int NW>
struct BatchSmem {
    static constexpr size_t body = (StepSmem<C, P, CX, CY, CZ, NW>::bytes + 15) / 16 * 16;
    static constexpr size_t tab = (sizeof(StepTables<C, P>) + 15) / 16 * 16;
    static constexpr size_t arg = (sizeof(StepArgs) + 15) / 16 * 16;
    static constexpr size_t bytes = body + tab + arg;
};

template <typename C, int P, int CX, int CY, int CZ, int NW>
__global__ void __launch_bounds__(NW * 32)
    batch_step_kernel(const BatchJob* __restrict__ jobs, int njobs, const StepTables<C, P>* __restrict__ tabs,
                      long long total, int parity, const __grid_constant__ Lattice<C> lat) {
    using BS = BatchSmem<C, P, CX, CY, CZ, NW>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepTables<C, P>* st = reinterpret_cast<StepTables<C, P>*>(smem_raw + BS::body);
    StepArgs* sa = reinterpret_cast<StepArgs*>(smem_raw + BS::body + BS::tab);
    int have = -1;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].tile_begin <= w) lo = mid;
            else hi = mid - 1;
        }
        if (lo != have) {
            static_assert(sizeof(StepTables<C, P>) % 4 == 0, "tables are copied in 4-byte words");
            const unsigned* tsrc = reinterpret_cast<const unsigned*>(tabs + lo);
            unsigned* tdst = reinterpret_cast<unsigned*>(st);
            for (int k = threadIdx.x; k < static_cast<int>(sizeof(StepTables<C, P>) / 4); k += NW * 32)
                tdst[k] = tsrc[k];
            if (threadIdx.x == 0) *sa = jobs[lo].args[parity];
            have = lo;
            __syncthreads();
        }
        LatticeCollideOp<C, P> op{lat};
        step_tile<C, C, P, CX, CY, CZ, NW, false>(*sa, *st, static_cast<int>(w - jobs[lo].tile_begin), smem_raw, op);
        __syncthreads();  // the next item reuses the shared memory
    }
}

// Launches step_kernel<..., PR, KC> over the tiles [q] of a launch (helper of launch_step_tiled).
template <typename S, typename C, int P, int CX, int CY, int CZ, int NW, bool PR, bool KC>
cudaError_t launch_step_variant(const StepArgs& args, const StepTables<C, P>& tab, long long ntiles,
                                cudaStream_t stream) {
    using SM = StepSmem<C, P, CX, CY, CZ, NW>;
    auto k = step_kernel<S, C, P, CX, CY, CZ, NW, PR, KC>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SM::bytes));
    if (err == cudaSuccess) {
        k<<<static_cast<unsigned>(ntiles), NW * 32, SM::bytes, stream>>>(args, tab);
        err = cudaGetLastError();
    }
    return err;
}

// WITH_PR = false instantiates only the kernel without the Prandtl term (tile-shape
// variants offered to the autotuner); such a launcher refuses contexts with the term on.
// WITH_KC = true also instantiates the compensated-moment kernels (FP32 arithmetic); a
// launcher without them refuses a context that asks for compensation, and FP64 arithmetic
// ignores the request (its sums need none).
template <typename S, typename C, int P, int CX, int CY, int CZ, int NW, bool WITH_PR = true, bool WITH_KC = true>
int launch_step_tiled(sllbm_ctx* ctx, const void* src, void* dst) {
    if (!WITH_PR && ctx->prm.pr_correction) return SLLBM_EINVAL;
    constexpr bool kKC = WITH_KC && sizeof(C) == 4;
    if (!WITH_KC && sizeof(C) == 4 && ctx->compensated) return SLLBM_EINVAL;
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
    if (static_cast<long long>(args.tiles[0]) * args.tiles[1] * args.tiles[2] > 0x7fffffffLL) return SLLBM_EINVAL;
    // all z-tiles, or the part of a slab's tiles its split step asks for
    int ranges[2][2];
    const int nr = slab_tile_ranges(ctx, CZ, ranges);
    cudaError_t err = cudaSuccess;
    for (int q = 0; q < nr && err == cudaSuccess; ++q) {
        args.tz_begin = ranges[q][0];
        const long long ntiles =
            static_cast<long long>(args.tiles[0]) * args.tiles[1] * (ranges[q][1] - ranges[q][0]);
        if (ntiles <= 0) continue;
        const bool kc = kKC && ctx->compensated;
        if (ctx->prm.pr_correction) {
            if constexpr (WITH_PR) {
                if constexpr (kKC) {
                    if (kc) err = launch_step_variant<S, C, P, CX, CY, CZ, NW, true, true>(args, *tab, ntiles, ctx->stream);
                }
                if (!kc) err = launch_step_variant<S, C, P, CX, CY, CZ, NW, true, false>(args, *tab, ntiles, ctx->stream);
            }
        } else {
            if constexpr (kKC) {
                if (kc) err = launch_step_variant<S, C, P, CX, CY, CZ, NW, false, true>(args, *tab, ntiles, ctx->stream);
            }
            if (!kc) err = launch_step_variant<S, C, P, CX, CY, CZ, NW, false, false>(args, *tab, ntiles, ctx->stream);
        }
        ctx->launches += 1;
    }
    if (err != cudaSuccess) {
        ctx->last_err = static_cast<int>(err);
        return SLLBM_ECUDA;
    }
    return SLLBM_OK;
}

}  // namespace sllbm
