// First pass on 8-bit input, exact: integer window sums (exact in float32 below
// 2^24), selection by int64 cross-multiplication, correctly rounded S_m / n_m.
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd_u8(int R, bool tie_app, const FwdParams &p, dim3 grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                       \
    case RR:                                                                                \
        return tie_app ? launch_fwd_tile<uint8_t, float, RR, true, true, true>(p, grid, s) \
                       : launch_fwd_tile<uint8_t, float, RR, false, true, true>(p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace osbf
