// Persistent TMA-fed forward kernels, f16 storage.
#include "fwd2_dispatch.cuh"

namespace osbf {

cudaError_t launch_fwd2_f16(int R, bool tie_app, bool maps, bool direct, const CUtensorMap &src,
                           const v2::Fwd2Params &p, int grid, cudaStream_t s) {
    return launch_fwd2_t<__half, false>(R, tie_app, maps, direct, src, p, grid, s);
}

int occupancy_fwd2_f16(int R, bool tie_app, bool maps, bool direct, int D) {
    return occupancy_fwd2_t<__half, false>(R, tie_app, maps, direct, D);
}

size_t smem_fwd2_f16(int R, int D, bool direct) { return (size_t)v2::make_layout2<__half>(R, D, direct).bytes; }

}  // namespace osbf
