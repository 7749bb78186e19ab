// BF16 tensor-core form of the network sweeps (tcgen05, sm_103a).
#include <cuda_runtime.h>

#include "internal.cuh"

namespace fbsde {

struct Bf16Work {
    int unused;
};

fbsde_status bf16_create(fbsde_ctx* ctx) {
    return set_err(ctx, FBSDE_ERR_UNSUPPORTED, "BF16 form not built yet");
}
void bf16_destroy(fbsde_ctx* ctx) { ctx->bf = nullptr; }
fbsde_status bf16_prepare_weights(fbsde_ctx* ctx, const float*) { return set_err(ctx, FBSDE_ERR_UNSUPPORTED, "BF16"); }
fbsde_status bf16_forward(fbsde_ctx* ctx, const float*) { return set_err(ctx, FBSDE_ERR_UNSUPPORTED, "BF16"); }
fbsde_status bf16_backward(fbsde_ctx* ctx, const float*, float*) { return set_err(ctx, FBSDE_ERR_UNSUPPORTED, "BF16"); }

}  // namespace fbsde
