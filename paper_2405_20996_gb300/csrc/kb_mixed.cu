// Mixed-precision path (FP32 gather, 3xTF32 tcgen05 contraction); filled in later.
#include "kb_internal.h"

kb_status kb_bubble_mixed(kb_ctx* ctx, int, int, int, int, int, unsigned, double, double, cudaStream_t) {
    ctx->err = "mixed precision path not built yet";
    return KB_ERR_UNSUPPORTED;
}
