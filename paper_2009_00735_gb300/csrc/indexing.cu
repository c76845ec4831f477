// indexing.cu -- steps (a6) look-up-table matching (Eq. 3) and (a7)
// Gauss-Newton orientation refinement.  Entry points are wired; kernels land next.
#include "common.cuh"

using namespace aptidx;

extern "C" {

int aptidx_set_reference(aptidx_ctx* ctx, int32_t, const float*, int32_t, const float*, int) {
    if (!ctx) return APTIDX_E_INVALID_ARG;
    return set_error(&ctx->c, APTIDX_E_INVALID_ARG, "set_reference: not built yet");
}
int aptidx_build_lut(aptidx_ctx* ctx, int32_t, const double*, int64_t, int) {
    if (!ctx) return APTIDX_E_INVALID_ARG;
    return set_error(&ctx->c, APTIDX_E_INVALID_ARG, "build_lut: not built yet");
}
int aptidx_match(aptidx_ctx* ctx, int32_t, const float*, int64_t, int32_t*, float*, int) {
    if (!ctx) return APTIDX_E_INVALID_ARG;
    return set_error(&ctx->c, APTIDX_E_INVALID_ARG, "match: not built yet");
}
int aptidx_refine_loss(aptidx_ctx* ctx, int32_t, const float*, const double*, int64_t, float*, float*, int) {
    if (!ctx) return APTIDX_E_INVALID_ARG;
    return set_error(&ctx->c, APTIDX_E_INVALID_ARG, "refine_loss: not built yet");
}
int aptidx_refine(aptidx_ctx* ctx, int32_t, const float*, const double*, int64_t, int32_t, double*, float*, int) {
    if (!ctx) return APTIDX_E_INVALID_ARG;
    return set_error(&ctx->c, APTIDX_E_INVALID_ARG, "refine: not built yet");
}

}  // extern "C"
