// FP32 storage / FP32 arithmetic instances of the fused step kernel.
#include "step_kernel.cuh"

namespace sllbm {

int launch_step_f32(sllbm_ctx* ctx, const void* src, void* dst) {
    switch (ctx->p) {
    case 2: return launch_step_tiled<float, float, 2, 4, 4, 2, 10>(ctx, src, dst);
    case 3: return launch_step_tiled<float, float, 3, 2, 2, 2, 10>(ctx, src, dst);
    case 4: return launch_step_tiled<float, float, 4, 2, 2, 1, 10>(ctx, src, dst);
    }
    return SLLBM_EINVAL;
}

}  // namespace sllbm
