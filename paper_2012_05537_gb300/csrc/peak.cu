// Arithmetic-peak microbenchmark of the library (the paper has no counterpart): the FP32,
// packed FP32x2 and FP64 fused multiply-add rates of the current GPU, measured with the
// same kind of instruction the step kernels use, so that a step's arithmetic can be set
// against a measured ALU roofline rather than a nominal one.
//
// Every thread runs kChains independent dependent chains a <- a*m + c (m, c kernel
// arguments, so nothing folds; the chains converge to c/(1-m) and stay finite), with
// enough resident warps per SM sub-partition to hide the FMA latency.  The result goes to
// a file-scope device word only if it equals a value it never takes, which keeps the
// arithmetic alive without any allocation.
#include <cuda_runtime.h>

#include "packed.cuh"
#include "sllbm.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kBlock = 512;

__device__ float g_peak_sink_f;
__device__ double g_peak_sink_d;

template <int KIND>  // 0: FP32 fma.rn.f32, 1: FP32x2 fma.rn.f32x2, 2: FP64 fma.rn.f64
__global__ void __launch_bounds__(kBlock) fma_peak_kernel(int iters, double m, double c) {
    if constexpr (KIND == 2) {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 0.5 * k + threadIdx.x * 1e-3;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == -1.0) g_peak_sink_d = s;
    } else if constexpr (KIND == 1) {
        const float2 mm = make_float2(static_cast<float>(m), static_cast<float>(m));
        const float2 cc = make_float2(static_cast<float>(c), static_cast<float>(c));
        float2 a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = make_float2(0.5f * k + threadIdx.x * 1e-3f, 0.25f * k);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = sllbm::ffma2(a[k], mm, cc);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
        if (s == -1.0f) g_peak_sink_f = s;
    } else {
        const float mm = static_cast<float>(m), cc = static_cast<float>(c);
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 0.5f * k + threadIdx.x * 1e-3f;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], mm, cc);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == -1.0f) g_peak_sink_f = s;
    }
}

template <int KIND>
cudaError_t launch_peak(int grid, int iters, cudaStream_t s) {
    fma_peak_kernel<KIND><<<grid, kBlock, 0, s>>>(iters, 0.9999, 1e-4);
    return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int grid, int iters, cudaStream_t s) {
    return kind == 0 ? launch_peak<0>(grid, iters, s) : kind == 1 ? launch_peak<1>(grid, iters, s)
                                                                  : launch_peak<2>(grid, iters, s);
}

}  // namespace

extern "C" int sllbm_fma_peak(int kind, int iters, void* cuda_stream, double* flops_per_s, double* seconds) {
    if (kind < 0 || kind > 2 || iters < 1 || flops_per_s == nullptr) return SLLBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLLBM_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SLLBM_ECUDA;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return SLLBM_ECUDA;
    const int grid = sms * (per_sm / kBlock > 0 ? per_sm / kBlock : 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return SLLBM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SLLBM_ECUDA;
    }
    cudaError_t e = launch_kind(kind, grid, iters, s);  // warm-up (clocks, module load)
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_kind(kind, grid, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.f)) return SLLBM_ECUDA;
    const double lanes = kind == 1 ? 2.0 : 1.0;  // FMAs per thread instruction
    const double fmas = static_cast<double>(grid) * kBlock * kChains * kUnroll * static_cast<double>(iters) * lanes;
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    if (seconds != nullptr) *seconds = ms * 1e-3;
    return SLLBM_OK;
}
