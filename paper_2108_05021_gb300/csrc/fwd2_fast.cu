// Single-pass kernels of the fast approximation (Sec. "Fast Approximation to One-sided
// Box Filter", Algorithm 3, Eq. (app)): float32 frames, paper tie order, results (and,
// with maps, selections) written from registers straight into the destination.
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd2_fast(int R, bool maps, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                             cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                         \
    case RR:                                                                                  \
        return maps ? v2::launch_fwd2<float, RR, false, true, true, true>(src, p, grid, s)   \
                    : v2::launch_fwd2<float, RR, false, false, true, true>(src, p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

int occupancy_fwd2_fast(int R, bool maps) {
    switch (R) {
#define OSBF_CASE(RR)                                                                 \
    case RR:                                                                          \
        return maps ? v2::occupancy_fwd2<float, RR, false, true, true, true>(1)      \
                    : v2::occupancy_fwd2<float, RR, false, false, true, true>(1);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return 0;
}

}  // namespace osbf
