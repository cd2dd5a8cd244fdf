// osbf_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "osbf_fwd.cuh"
#include "osbf_fwd2.cuh"

// every radius with a compiled kernel
#define OSBF_FOR_EACH_R(X) \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

namespace osbf {

enum class Storage { F32 = 0, F16 = 1, BF16 = 2, U8 = 3 };

// row pitch (bytes) of the selection maps: frame width rounded up to 16 bytes
inline int maps_pitch(int FW) { return (FW + 15) / 16 * 16; }

// The exact first pass on 8-bit input (the first-pass tile kernel of osbf_fwd.cuh).
cudaError_t launch_fwd_u8(int R, bool tie_app, const FwdParams &p, dim3 grid, cudaStream_t s);

// dynamic shared memory of one forward CTA (first-pass kernel)
size_t fwd_smem(Storage st, int R, int D);

// persistent TMA-fed forward (frames in, frame or cropped output out)
cudaError_t launch_fwd2_f32(int R, bool tie_app, bool maps, bool direct, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                            cudaStream_t s);
cudaError_t launch_fwd2_f16(int R, bool tie_app, bool maps, bool direct, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                            cudaStream_t s);
cudaError_t launch_fwd2_bf16(int R, bool tie_app, bool maps, bool direct, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                             cudaStream_t s);
int occupancy_fwd2_f32(int R, bool tie_app, bool maps, bool direct, int D);
int occupancy_fwd2_f16(int R, bool tie_app, bool maps, bool direct, int D);
int occupancy_fwd2_bf16(int R, bool tie_app, bool maps, bool direct, int D);
size_t smem_fwd2_f32(int R, int D, bool direct);
size_t smem_fwd2_f16(int R, int D, bool direct);
size_t smem_fwd2_bf16(int R, int D, bool direct);

// the fast approximation, single pass per launch (float32, paper tie order)
cudaError_t launch_fwd2_fast(int R, bool maps, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                             cudaStream_t s);
int occupancy_fwd2_fast(int R, bool maps);

// single-pass float32 launches of the appendix tie order (results and selections staged)
cudaError_t launch_fwd2_app_f32(int R, bool maps, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                                cudaStream_t s);
int occupancy_fwd2_app_f32(int R, bool maps);

// single-pass float32 launches with per-warp tensor stores (R % 4 == 0, paper tie order, no maps)
// padin: the first pass straight from the unpadded image (replicate pad in the kernel)
cudaError_t launch_fwd2_tstore(int R, bool fast, const CUtensorMap &src, const CUtensorMap &dmap,
                               const v2::Fwd2Params &p, int grid, cudaStream_t s, bool padin = false);
int occupancy_fwd2_tstore(int R, bool fast);
// single-pass float32 frame-to-frame launches that issue the next tile's load before pass H
// (R % 4 == 0, paper tie order, no maps; 32-byte register stores into a frame whose row
// pitch is a multiple of 32 floats)
cudaError_t launch_fwd2_early(int R, bool fast, const CUtensorMap &src, const v2::Fwd2Params &p, int grid,
                              cudaStream_t s);
int occupancy_fwd2_early(int R, bool fast);
// The radii whose frame-to-frame passes take the early-load kernel: at r = 8, 12, 16 it is
// 2-6 % faster than the tensor-store kernel on 4096^2 x 3 planes; at r = 4 0.7 % slower.
inline bool fwd2_early_radius(int r) { return r % 4 == 0 && r >= 8; }

// A float32 destination for tensor stores: P planes of H rows x W elements (row pitch
// `pitch` elements), 32 x 32 boxes staged with the 128-byte swizzle.
bool encode_store_map(CUtensorMap *map, void *base, int W, int H, int P, int pitch);

bool encode_frame_map(CUtensorMap *map, Storage st, const void *base, int FW, int FH, int P, int pitch, int box_w,
                      int box_h);
cudaError_t launch_pad_replicate(Storage st, const void *in, void *frame, int P, int H, int W, int R, int FH, int FW,
                                 int FWp, cudaStream_t s);

// One launch of the forward (D fused passes) from a padded frame into a frame or the
// caller's cropped output, with the kernel variant every entry point uses (osbf_api.cu).
struct GroupLaunch {
    Storage st = Storage::F32;
    int r = 0, D = 1, tie = 0;
    const void *src = nullptr;  // padded frame, row pitch src_pitch elements
    int src_pitch = 0;
    void *dst = nullptr;  // frame (row pitch dst_pitch) or, with dst_is_output, the H x W output
    int dst_pitch = 0;
    int dst_is_output = 0;
    int P = 0, H = 0, W = 0;
    uint8_t *maps = nullptr;  // optional selection maps (osbf_filter_ex layout)
    int map_iter0 = 0;
    long long map_iter_stride = 0;
    unsigned int *err = nullptr;  // device error word
    int sms = 0;
    int variant = 0;  // forward kernel: 0 = library choice, 1 = tile kernel, 2 = streaming strip kernel
    int src_is_image = 0;  // src is the caller's unpadded image (row pitch W): the first pass pads it itself
    int fast = 0;  // the fast approximation (float32, paper tie order, single passes written from registers)
};
cudaError_t launch_group(const GroupLaunch &g, cudaStream_t s, const char **what);

// streaming strip forward (osbf_strip.cuh, fwd2_strip.cu): float32, one pass per launch,
// paper tie order, radii 1..OSBF_STRIP_MAX_R
#define OSBF_STRIP_MAX_R 8
namespace strip {
struct StripParams;
}
// v8: results leave from registers by 32-byte stores (r % 4 == 0, no maps, the destination's
// strip columns on 32 bytes); otherwise they are staged per warp and written row by row
cudaError_t launch_fwd_strip(int R, bool maps, bool v8, const CUtensorMap &src, const strip::StripParams &sp,
                             int grid, cudaStream_t s);
int occupancy_fwd_strip(int R, bool maps, bool v8);
int strip_box_width(int R);

// the final crop of a float32 frame into H x W planes (osbf_misc.cu)
cudaError_t launch_crop_f32(const float *frame, float *out, int P, int H, int W, int R, int FWp, cudaStream_t s);
// the same for 16-bit storage (FWp in elements)
cudaError_t launch_crop_16(const void *frame, void *out, int P, int H, int W, int R, int FWp, cudaStream_t s);

// elementwise helpers (osbf_misc.cu)
cudaError_t launch_u8_to_f32(const uint8_t *in, float *out, long long n, cudaStream_t s);
cudaError_t launch_fill_u8(uint8_t *p, uint8_t v, long long n, cudaStream_t s);
// a non-constant synthetic image (P planes of H x W) in the given storage type, for tuning
cudaError_t launch_tuning_image(Storage st, void *p, int P, int H, int W, cudaStream_t s);

}  // namespace osbf
