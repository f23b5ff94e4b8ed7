// FP32 storage / FP32 arithmetic step: the TMA-fed persistent kernel (step_tma.cu) where
// the mesh allows it and the context selects it, the generic tile kernel (step_kernel.cuh)
// otherwise.
#include "step_kernel.cuh"

namespace sllbm {

int launch_step_f32(sllbm_ctx* ctx, const void* src, void* dst) {
    if (ctx->step_kernel == 2) return launch_step_tma(ctx, src, dst);
    if (ctx->tile_shape != 0) return launch_step_f32_shape(ctx, src, dst, ctx->tile_shape);
    // p = 3: tiles of 4x2x1 cells with 9 warps fit twice on an SM (shared memory, and
    // registers capped for two CTAs), so one CTA's collision overlaps another's streaming, and
    // the 45 velocity pairs split evenly over the warps; measured about 8 % faster than 2x2x2
    // cells with 16 warps (4 % from the second CTA, 4 % from the even split).  At p = 2 and
    // p = 4 the two-CTA shapes tried were slower.
    switch (ctx->p) {
    case 2: return launch_step_tiled<float, float, 2, 4, 4, 2, 16>(ctx, src, dst);
    case 3: return launch_step_tiled<float, float, 3, 4, 2, 1, 9>(ctx, src, dst);
    case 4: return launch_step_tiled<float, float, 4, 2, 2, 1, 16>(ctx, src, dst);
    }
    return SLLBM_EINVAL;
}

}  // namespace sllbm
