// Radius / variant dispatch of the persistent forward kernel (osbf_fwd2.cuh), shared by
// the per-storage-type translation units (fwd2_f32.cu, fwd2_f16.cu, fwd2_bf16.cu).
//   direct : one pass per launch written from registers into the destination
//            (paper tie order; float32 also the appendix order, fwd2_app.cu; with or
//            without maps)
//   general: fused passes through shared memory (both tie orders; maps for the
//            appendix order only where APP_MAPS)
#pragma once

#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

namespace osbf {

// direct float32 kernels stage their results per warp and write them a row at a time
template <typename T> constexpr bool kStage = sizeof(T) == 4;
// direct 16-bit kernels without maps widen their box in pass V and load the next tile
// before pass H (osbf_fwd2.cuh, EARLY)
template <typename T> constexpr bool kEarly = sizeof(T) == 2;

template <typename T, bool APP_MAPS>
cudaError_t launch_fwd2_t(int R, bool tie_app, bool maps, bool direct, const CUtensorMap &src,
                          const v2::Fwd2Params &p, int grid, cudaStream_t s) {
    if (direct && tie_app) {  // float32 only (fwd2_app.cu)
        if constexpr (sizeof(T) == 4) return launch_fwd2_app_f32(R, maps, src, p, grid, s);
        return cudaErrorInvalidValue;
    }
    switch (R) {
#define OSBF_CASE(RR)                                                                                    \
    case RR:                                                                                             \
        if (direct && !tie_app)                                                                          \
            return maps ? v2::launch_fwd2<T, RR, false, true, true, false, false, kStage<T>>(src, p, grid, s) \
                        : v2::launch_fwd2<T, RR, false, false, true, false, false, kStage<T>, false, kEarly<T>>(src, p, grid, s); \
        if (tie_app) {                                                                                   \
            if (!maps) return v2::launch_fwd2<T, RR, true, false, false>(src, p, grid, s);               \
            if constexpr (APP_MAPS) return v2::launch_fwd2<T, RR, true, true, false>(src, p, grid, s);   \
            return cudaErrorInvalidValue;                                                                \
        }                                                                                                \
        return maps ? v2::launch_fwd2<T, RR, false, true, false>(src, p, grid, s)                        \
                    : v2::launch_fwd2<T, RR, false, false, false>(src, p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename T, bool APP_MAPS>
int occupancy_fwd2_t(int R, bool tie_app, bool maps, bool direct, int D) {
    if (direct && tie_app) {
        if constexpr (sizeof(T) == 4) return occupancy_fwd2_app_f32(R, maps);
        return 0;
    }
    switch (R) {
#define OSBF_CASE(RR)                                                                     \
    case RR:                                                                              \
        if (direct && !tie_app)                                                           \
            return maps ? v2::occupancy_fwd2<T, RR, false, true, true, false, false, kStage<T>>(D) \
                        : v2::occupancy_fwd2<T, RR, false, false, true, false, false, kStage<T>, kEarly<T>>(D); \
        if (tie_app) {                                                                    \
            if (!maps) return v2::occupancy_fwd2<T, RR, true, false, false>(D);           \
            if constexpr (APP_MAPS) return v2::occupancy_fwd2<T, RR, true, true, false>(D); \
            return 0;                                                                     \
        }                                                                                 \
        return maps ? v2::occupancy_fwd2<T, RR, false, true, false>(D)                    \
                    : v2::occupancy_fwd2<T, RR, false, false, false>(D);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return 0;
}

}  // namespace osbf
