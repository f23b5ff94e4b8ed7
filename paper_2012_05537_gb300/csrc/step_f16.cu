// 16-bit deviation storage (IEEE half, bfloat16) / FP32 arithmetic: the TMA-fed kernel
// (step_tma.cu) where the mesh allows it and the context selects it, the generic tile
// kernel otherwise.
#include "step_kernel.cuh"

namespace sllbm {

template <typename S>
int launch_step_dev(sllbm_ctx* ctx, const void* src, void* dst) {
    // the tile shapes of the FP32 instances (p = 3: two 9-warp CTAs per SM)
    switch (ctx->p) {
    case 2: return launch_step_tiled<S, float, 2, 4, 4, 2, 16>(ctx, src, dst);
    case 3: return launch_step_tiled<S, float, 3, 4, 2, 1, 9>(ctx, src, dst);
    case 4: return launch_step_tiled<S, float, 4, 2, 2, 1, 16>(ctx, src, dst);
    }
    return SLLBM_EINVAL;
}

int launch_step_f16(sllbm_ctx* ctx, const void* src, void* dst) {
    if (ctx->step_kernel == 2) return launch_step_tma(ctx, src, dst);
    if (ctx->prm.storage == SLLBM_BF16DEV) return launch_step_dev<__nv_bfloat16>(ctx, src, dst);
    return launch_step_dev<__half>(ctx, src, dst);
}

}  // namespace sllbm
