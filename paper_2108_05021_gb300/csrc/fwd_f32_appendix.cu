// Forward kernels, float32 storage, the appendix's tie order (N6 N5 N7 N8 N2 N1 N3 N4).
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd_f32_appendix(int R, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                        \
    case RR:                                                                                 \
        return maps ? launch_fwd_tile<float, float, RR, true, true, false>(p, grid, s)      \
                    : launch_fwd_tile<float, float, RR, true, false, false>(p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace osbf
