// Forward kernels, f16 storage: window sums and scores in float32, every pass's
// result rounded to f16 before the next pass reads it.
// Selection maps are written with the paper's tie order only.
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd_f16(int R, bool tie_app, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                  \
    case RR:                                                                           \
        return tie_app ? launch_fwd_tile<__half, __half, RR, true, false, false>(p, grid, s)       \
                       : (maps ? launch_fwd_tile<__half, __half, RR, false, true, false>(p, grid, s)  \
                               : launch_fwd_tile<__half, __half, RR, false, false, false>(p, grid, s));
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace osbf
