// Forward kernels, bf16 storage: window sums and scores in float32, every pass's
// result rounded to bf16 before the next pass reads it.
// Selection maps are written with the paper's tie order only.
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd_bf16(int R, bool tie_app, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                  \
    case RR:                                                                           \
        return tie_app ? launch_fwd_tile<__nv_bfloat16, __nv_bfloat16, RR, true, false, false>(p, grid, s)       \
                       : (maps ? launch_fwd_tile<__nv_bfloat16, __nv_bfloat16, RR, false, true, false>(p, grid, s)  \
                               : launch_fwd_tile<__nv_bfloat16, __nv_bfloat16, RR, false, false, false>(p, grid, s));
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace osbf
