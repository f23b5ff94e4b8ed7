// Population storage types of the library (device side).
//
// SLLBM_F64 and SLLBM_F32 store f_i and g_i themselves.  The 16-bit types (SLLBM_F16DEV,
// SLLBM_BF16DEV) store the deviations of the populations from the weights times the
// reference state (rho0, T0) of the context:
//
//     d_i  = f_i / w_i - rho0,        d_gi = g_i / w_i - (2 C_v - D) T0 rho0,
//
// which are O(Ma^2, T/T0 - 1) instead of spanning the four decades of the weights, so a
// 16-bit mantissa holds them with useful relative accuracy.  The Lagrange weights of a pass
// sum to one, so interpolating the deviations gives the deviations of the interpolated
// populations: the streaming operates on the stored values directly (in FP32).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sllbm {

// Deviation references per population kind: ref_f = rho0, ref_g = (2 C_v - D) T0 rho0.
struct PopRef {
    double f, g;
};

template <typename S>
struct PopCodec {
    static constexpr bool kDev = false;
    __device__ __forceinline__ static double decode(S v, double, double) { return static_cast<double>(v); }
    __device__ __forceinline__ static S encode(double x, double, double) { return static_cast<S>(x); }
};

template <>
struct PopCodec<__half> {
    static constexpr bool kDev = true;
    __device__ __forceinline__ static double decode(__half v, double w, double ref) {
        return w * (static_cast<double>(__half2float(v)) + ref);
    }
    __device__ __forceinline__ static __half encode(double x, double w, double ref) {
        return __float2half_rn(static_cast<float>(x / w - ref));
    }
};

template <>
struct PopCodec<__nv_bfloat16> {
    static constexpr bool kDev = true;
    __device__ __forceinline__ static double decode(__nv_bfloat16 v, double w, double ref) {
        return w * (static_cast<double>(__bfloat162float(v)) + ref);
    }
    __device__ __forceinline__ static __nv_bfloat16 encode(double x, double w, double ref) {
        return __float2bfloat16_rn(static_cast<float>(x / w - ref));
    }
};

}  // namespace sllbm
