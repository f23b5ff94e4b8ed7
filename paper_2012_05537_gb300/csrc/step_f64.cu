// FP64 storage / FP64 arithmetic instances of the fused step kernel.
#include "step_kernel.cuh"

namespace sllbm {

int launch_step_f64(sllbm_ctx* ctx, const void* src, void* dst) {
    switch (ctx->p) {
    case 2: return launch_step_tiled<double, double, 2, 4, 2, 2, 8>(ctx, src, dst);
    case 3: return launch_step_tiled<double, double, 3, 2, 2, 1, 8>(ctx, src, dst);
    case 4: return launch_step_tiled<double, double, 4, 2, 1, 1, 8>(ctx, src, dst);
    }
    return SLLBM_EINVAL;
}

}  // namespace sllbm
