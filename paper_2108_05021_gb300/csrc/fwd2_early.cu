// Single-pass float32 frame-to-frame kernels that issue the next tile's load before pass H
// (osbf_fwd2.cuh, EARLY): radii that are multiples of 4, paper tie order, no maps; the exact
// filter and the fast approximation.
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd2_early(int R, bool fast, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                              cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                                        \
    case RR:                                                                                                 \
        return fast ? v2::launch_fwd2<float, RR, false, false, true, true, false, false, false, true>(src, p, grid, s) \
                    : v2::launch_fwd2<float, RR, false, false, true, false, false, false, false, true>(src, p, grid, s);
        OSBF_CASE(4) OSBF_CASE(8) OSBF_CASE(12) OSBF_CASE(16)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

int occupancy_fwd2_early(int R, bool fast) {
    switch (R) {
#define OSBF_CASE(RR)                                                                                   \
    case RR:                                                                                            \
        return fast ? v2::occupancy_fwd2<float, RR, false, false, true, true, false, false, true>(1)    \
                    : v2::occupancy_fwd2<float, RR, false, false, true, false, false, false, true>(1);
        OSBF_CASE(4) OSBF_CASE(8) OSBF_CASE(12) OSBF_CASE(16)
#undef OSBF_CASE
    }
    return 0;
}

}  // namespace osbf
