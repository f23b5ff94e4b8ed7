// Alternative tile shapes of the generic FP32 step kernel, offered to the autotuner
// (sllbm_autotune): smaller tiles give more CTAs (and more CTAs per SM) on small meshes,
// at the price of more re-read halo per node.  Without the Prandtl term only.
#include "step_kernel.cuh"

namespace sllbm {

int launch_step_f32_shape(sllbm_ctx* ctx, const void* src, void* dst, int shape) {
    if (shape == 1) {
        switch (ctx->p) {
        case 2: return launch_step_tiled<float, float, 2, 4, 2, 2, 16, false>(ctx, src, dst);
        case 3: return launch_step_tiled<float, float, 3, 2, 2, 1, 16, false>(ctx, src, dst);
        case 4: return launch_step_tiled<float, float, 4, 2, 1, 1, 16, false>(ctx, src, dst);
        }
    } else if (shape == 2) {
        switch (ctx->p) {
        case 2: return launch_step_tiled<float, float, 2, 2, 2, 1, 8, false>(ctx, src, dst);
        case 3: return launch_step_tiled<float, float, 3, 1, 1, 1, 8, false>(ctx, src, dst);
        case 4: return launch_step_tiled<float, float, 4, 1, 1, 1, 8, false>(ctx, src, dst);
        }
    }
    return SLLBM_EINVAL;
}

}  // namespace sllbm
