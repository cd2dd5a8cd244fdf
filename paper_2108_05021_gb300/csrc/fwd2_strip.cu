// Streaming strip forward kernels (osbf_strip.cuh): float32, one pass per launch, paper
// tie order, radii 1..OSBF_STRIP_MAX_R.
#include "osbf_internal.h"
#include "osbf_strip.cuh"

namespace osbf {

namespace {

template <int R>
cudaError_t launch_r(bool maps, bool v8, const CUtensorMap &src, const strip::StripParams &sp, int grid,
                     cudaStream_t s) {
    if constexpr (R % 4 == 0)
        if (v8 && !maps) return strip::launch_strip<R, false, true>(src, sp, grid, s);
    if (v8) return cudaErrorInvalidValue;
    return maps ? strip::launch_strip<R, true, false>(src, sp, grid, s)
                : strip::launch_strip<R, false, false>(src, sp, grid, s);
}

template <int R>
int occupancy_r(bool maps, bool v8) {
    if constexpr (R % 4 == 0)
        if (v8 && !maps) return strip::occupancy_strip<R, false, true>();
    if (v8) return 0;
    return maps ? strip::occupancy_strip<R, true, false>() : strip::occupancy_strip<R, false, false>();
}

}  // namespace

cudaError_t launch_fwd_strip(int R, bool maps, bool v8, const CUtensorMap &src, const strip::StripParams &sp,
                             int grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR) \
    case RR: return launch_r<RR>(maps, v8, src, sp, grid, s);
        OSBF_CASE(1) OSBF_CASE(2) OSBF_CASE(3) OSBF_CASE(4) OSBF_CASE(5) OSBF_CASE(6) OSBF_CASE(7) OSBF_CASE(8)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

int occupancy_fwd_strip(int R, bool maps, bool v8) {
    switch (R) {
#define OSBF_CASE(RR) \
    case RR: return occupancy_r<RR>(maps, v8);
        OSBF_CASE(1) OSBF_CASE(2) OSBF_CASE(3) OSBF_CASE(4) OSBF_CASE(5) OSBF_CASE(6) OSBF_CASE(7) OSBF_CASE(8)
#undef OSBF_CASE
    }
    return 0;
}

int strip_box_width(int R) { return strip::make_strip_layout(R, false, true).PU; }

}  // namespace osbf
