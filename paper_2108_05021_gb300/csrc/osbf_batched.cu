// Batched persistent launch (placeholder until the persistent kernel lands).
#include "osbf.h"
#include "osbf_internal.h"

osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg);

void osbf_batched_free(osbf_ctx *) {}

extern "C" osbf_status osbf_filter_batched(osbf_ctx *ctx, const osbf_job *, int, void *) {
    return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "batched launch not built yet");
}
