// Single-pass float32 kernels of the appendix tie order (osbf_fwd2.cuh with TIE_APP): the
// same sweep as the paper order's single-pass kernels, results (and, with maps, the
// selections) staged per warp and written a row at a time.  A translation unit of their
// own, so they compile beside the paper order's kernels.
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd2_app_f32(int R, bool maps, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                                cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                                  \
    case RR:                                                                                           \
        return maps ? v2::launch_fwd2<float, RR, true, true, true, false, false, true>(src, p, grid, s) \
                    : v2::launch_fwd2<float, RR, true, false, true, false, false, true>(src, p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

int occupancy_fwd2_app_f32(int R, bool maps) {
    switch (R) {
#define OSBF_CASE(RR)                                                                           \
    case RR:                                                                                    \
        return maps ? v2::occupancy_fwd2<float, RR, true, true, true, false, false, true>(1)    \
                    : v2::occupancy_fwd2<float, RR, true, false, true, false, false, true>(1);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return 0;
}

}  // namespace osbf
