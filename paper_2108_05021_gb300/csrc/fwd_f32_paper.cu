// Forward kernels, float32 storage, paper tie order (N1..N8).
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd_f32_paper(int R, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                         \
    case RR:                                                                                  \
        return maps ? launch_fwd_tile<float, float, RR, false, true, false>(p, grid, s)      \
                    : launch_fwd_tile<float, float, RR, false, false, false>(p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace osbf
