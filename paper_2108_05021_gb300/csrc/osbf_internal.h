// osbf_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "osbf_fwd.cuh"

// every radius with a compiled kernel
#define OSBF_FOR_EACH_R(X) \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

namespace osbf {

enum class Storage { F32 = 0, F16 = 1, BF16 = 2, U8 = 3 };

// One fused group of forward passes (D = p.D) on the tile grid `grid`.
cudaError_t launch_fwd_f32_paper(int R, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s);
cudaError_t launch_fwd_f32_appendix(int R, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s);
cudaError_t launch_fwd_f16(int R, bool tie_app, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s);
cudaError_t launch_fwd_bf16(int R, bool tie_app, bool maps, const FwdParams &p, dim3 grid, cudaStream_t s);
cudaError_t launch_fwd_u8(int R, bool tie_app, const FwdParams &p, dim3 grid, cudaStream_t s);

// dynamic shared memory of one forward CTA
size_t fwd_smem(Storage st, int R, int D);

// elementwise helpers (osbf_misc.cu)
cudaError_t launch_u8_to_f32(const uint8_t *in, float *out, long long n, cudaStream_t s);
cudaError_t launch_fill_u8(uint8_t *p, uint8_t v, long long n, cudaStream_t s);

}  // namespace osbf
