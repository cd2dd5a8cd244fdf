// Persistent TMA-fed forward kernels, f32 storage.
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

namespace osbf {

// direct: one pass per launch written straight to the destination frame (paper tie
// order, no maps); otherwise the general kernel.
cudaError_t launch_fwd2_f32(int R, bool tie_app, bool maps, bool direct, const CUtensorMap &src,
                           const v2::Fwd2Params &p, int grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR)                                                                           \
    case RR:                                                                                    \
        if (direct) return v2::launch_fwd2<float, RR, false, false, true>(src, p, grid, s);      \
        if (tie_app) return maps ? v2::launch_fwd2<float, RR, true, true, false>(src, p, grid, s) : v2::launch_fwd2<float, RR, true, false, false>(src, p, grid, s); \
        return maps ? v2::launch_fwd2<float, RR, false, true, false>(src, p, grid, s)            \
                    : v2::launch_fwd2<float, RR, false, false, false>(src, p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

int occupancy_fwd2_f32(int R, bool tie_app, bool maps, bool direct, int D) {
    switch (R) {
#define OSBF_CASE(RR)                                                                  \
    case RR:                                                                           \
        if (direct) return v2::occupancy_fwd2<float, RR, false, false, true>(D);        \
        if (tie_app) return v2::occupancy_fwd2<float, RR, true, false, false>(D);       \
        return maps ? v2::occupancy_fwd2<float, RR, false, true, false>(D)              \
                    : v2::occupancy_fwd2<float, RR, false, false, false>(D);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return 0;
}

size_t smem_fwd2_f32(int R, int D, bool direct) { return (size_t)v2::make_layout2<float>(R, D, direct).bytes; }

}  // namespace osbf
