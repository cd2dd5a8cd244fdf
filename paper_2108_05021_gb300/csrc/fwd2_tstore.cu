// Single-pass float32 kernels whose results leave through per-warp tensor stores
// (osbf_fwd2.cuh, TSTORE): radii that are multiples of 4, paper tie order, no maps; the
// exact filter and the fast approximation.
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

namespace osbf {

cudaError_t launch_fwd2_tstore(int R, bool fast, const CUtensorMap &src, const CUtensorMap &dmap,
                               const v2::Fwd2Params &p, int grid, cudaStream_t s, bool padin) {
    switch (R) {
#define OSBF_CASE(RR)                                                                                   \
    case RR:                                                                                            \
        if (padin)                                                                                      \
            return fast ? v2::launch_fwd2<float, RR, false, false, true, true, true, false, true>(src, p, grid, s, &dmap) \
                        : v2::launch_fwd2<float, RR, false, false, true, false, true, false, true>(src, p, grid, s, &dmap); \
        return fast ? v2::launch_fwd2<float, RR, false, false, true, true, true>(src, p, grid, s, &dmap) \
                    : v2::launch_fwd2<float, RR, false, false, true, false, true>(src, p, grid, s, &dmap);
        OSBF_CASE(4) OSBF_CASE(8) OSBF_CASE(12) OSBF_CASE(16)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

int occupancy_fwd2_tstore(int R, bool fast) {
    switch (R) {
#define OSBF_CASE(RR)                                                                 \
    case RR:                                                                          \
        return fast ? v2::occupancy_fwd2<float, RR, false, false, true, true, true>(1) \
                    : v2::occupancy_fwd2<float, RR, false, false, true, false, true>(1);
        OSBF_CASE(4) OSBF_CASE(8) OSBF_CASE(12) OSBF_CASE(16)
#undef OSBF_CASE
    }
    return 0;
}

}  // namespace osbf
