// Per-node moments, equilibrium and BGK collision of the SLLBM (device code).
#pragma once

#include "tables.h"

namespace sllbm {

// |xi_i|^2 of shell s of the cubature set (exact: 0, 3, 9, 15).
__host__ __device__ constexpr double shell_xi2(int s) {
    return s == 0 ? 0.0 : (s == 1 ? 3.0 : (s == 2 ? 9.0 : 15.0));
}

// Coefficients of the fourth-order Hermite equilibrium written as a quartic in
// s = xi.u on each velocity shell.  Contracting the App. A moments (T_ref = 1,
// th = T - 1) with the App. B tensors (c_s = 1) in closed form gives
//   f_i^eq / (w_i rho) = c0 + c1 s + c2 s^2 + s^3/6 + s^4/24,
//   c0 = 1 - u^2/2 + th(x2-3)/2 + u^4/8 + th u^2 (5-x2)/4 + th^2 (x2^2 - 10 x2 + 15)/8,
//   c1 = 1 - u^2/2 + th(x2-5)/2,
//   c2 = 1/2 - u^2/4 + th(x2-7)/4,
// with x2 = |xi_i|^2.  Only the symmetric, shell-dependent scalars are formed once per
// node (the reuse Sec. IV.B describes); per velocity the cost is one dot product and a
// Horner evaluation.
template <typename C>
struct EqCoef {
    C c0[4], c1[4], c2[4];
};

template <typename C>
__device__ __forceinline__ EqCoef<C> eq_coefficients(C usq, C th) {
    EqCoef<C> e;
    const C half = C(0.5), quarter = C(0.25), eighth = C(0.125);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const C x2 = C(shell_xi2(s));
        e.c0[s] = C(1) - half * usq + half * th * (x2 - C(3)) + eighth * usq * usq
                + quarter * th * usq * (C(5) - x2)
                + eighth * th * th * (x2 * x2 - C(10) * x2 + C(15));
        e.c1[s] = C(1) - half * usq + half * th * (x2 - C(5));
        e.c2[s] = half - quarter * usq + quarter * th * (x2 - C(7));
    }
    return e;
}

template <typename C>
__device__ __forceinline__ C eq_poly(const EqCoef<C>& e, int sh, C s) {
    return e.c0[sh] + s * (e.c1[sh] + s * (e.c2[sh] + s * (C(1.0 / 6.0) + s * C(1.0 / 24.0))));
}

// Sutherland law, Sec. III.C: mu/mu_inf = 1.4042 T^1.5 / (T + 0.40417).
template <typename C>
__device__ __forceinline__ C sutherland(C T) {
    return C(1.4042) * T * sqrt(T) / (T + C(0.40417));
}

// d ln(mu/mu_inf) / dT of the same law: 3/(2T) - 1/(T + 0.40417).
template <typename C>
__device__ __forceinline__ C sutherland_dlog(C T) {
    return C(1.5) / T - C(1) / (T + C(0.40417));
}

}  // namespace sllbm
