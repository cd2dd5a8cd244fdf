// Backward kernels (placeholder until the adjoint kernels land).
#include "osbf.h"
#include "osbf_internal.h"

osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg);

osbf_status osbf_backward_impl(osbf_ctx *ctx, const float *, float *, const uint8_t *, int, int, int, int, int,
                               cudaStream_t) {
    return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "backward not built yet");
}

extern "C" osbf_status osbf_filter_checkpointed(osbf_ctx *ctx, const float *, float *, float *, int, int, int, int,
                                                int, int, int, void *) {
    return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "checkpointed forward not built yet");
}
extern "C" osbf_status osbf_filter_backward_checkpointed(osbf_ctx *ctx, const float *, float *, const float *, int,
                                                         int, int, int, int, int, int, void *) {
    return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "checkpointed backward not built yet");
}
