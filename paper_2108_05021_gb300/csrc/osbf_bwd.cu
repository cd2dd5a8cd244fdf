// Backward of the One-Sided Box Filter: the transpose of the crop (embed into a zero
// ring), per-pass adjoint launches (osbf_bwd.cuh), the transpose of the appendix's
// replicate padding, and the checkpointed forward/backward.
#include <cstring>

#include "osbf.h"
#include "osbf_bwd.cuh"
#include "osbf_internal.h"

osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg);
void *osbf_ctx_workspace(osbf_ctx *ctx, int slot, size_t bytes, osbf_status *st);
void osbf_ctx_count_launches(osbf_ctx *ctx, int n);
void osbf_ctx_reset_launches(osbf_ctx *ctx);
osbf_status osbf_forward_run(osbf_ctx *ctx, const void *in, int in_is_frame, int in_pitch, void *out, int out_is_frame,
                             int out_pitch, int P, int H, int W, int r, int iters, osbf_dtype dtype, int depth,
                             int tie, uint8_t *maps, int maps_iter0, long long maps_iter_stride, cudaStream_t s);

namespace osbf {

static cudaError_t launch_bwd(int R, const CUtensorMap &gmap, const CUtensorMap &mmap, const bwd::BwdParams &p,
                              int grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR) \
    case RR: return bwd::launch_bwd_kernel<RR>(gmap, mmap, p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
}

static int occupancy_bwd(int R) {
    switch (R) {
#define OSBF_CASE(RR) \
    case RR: return bwd::occupancy_bwd_kernel<RR>();
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return 0;
}

// Transpose of the crop: grad_out (H x W) inside the frame, zero on the ring.
__global__ void embed_zero_kernel(const float *__restrict__ g, float *__restrict__ frame, int H, int W, int R, int FW,
                                  int FWp) {
    const int fy = blockIdx.y, plane = blockIdx.z;
    const int y = fy - R;
    const bool yin = (unsigned)y < (unsigned)H;
    const float *src = g + ((long long)plane * H + (yin ? y : 0)) * W;
    float *dst = frame + ((long long)plane * gridDim.y + fy) * FWp;
    for (int fx = blockIdx.x * blockDim.x + threadIdx.x; fx < FW; fx += gridDim.x * blockDim.x) {
        const int x = fx - R;
        dst[fx] = (yin && (unsigned)x < (unsigned)W) ? src[x] : 0.f;
    }
}

// Transpose of the replicate padding: each image pixel collects the gradient of every
// frame pixel that was copied from it (its own frame pixel, plus the ring for edge pixels).
__global__ void pad_adjoint_kernel(const float *__restrict__ g, float *__restrict__ out, int H, int W, int R, int FW,
                                   int gpitch) {
    const int y = blockIdx.y, plane = blockIdx.z;
    const int FH = H + 2 * R;
    const int fy0 = y == 0 ? 0 : y + R, fy1 = y == H - 1 ? FH - 1 : y + R;
    const float *gp = g + (long long)plane * FH * gpitch;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x) {
        const int fx0 = x == 0 ? 0 : x + R, fx1 = x == W - 1 ? FW - 1 : x + R;
        float acc = 0.f;
        for (int fy = fy0; fy <= fy1; ++fy)
            for (int fx = fx0; fx <= fx1; ++fx) acc += gp[(long long)fy * gpitch + fx];
        out[((long long)plane * H + y) * W + x] = acc;
    }
}

}  // namespace osbf

using namespace osbf;

unsigned int *osbf_ctx_err_word(osbf_ctx *ctx);
int osbf_ctx_sms(const osbf_ctx *ctx);

namespace {

int frame_pitch_f32(int FW) { return (FW + 31) / 32 * 32; }

// The backward passes t = t1-1 .. t0 (maps + t * stride), starting from `g` (the caller's
// grad_out when g_is_output, else the gradient frame gbuf[*cur]); the result lands in one
// of the two gradient frames, whose index is returned through *cur.
osbf_status run_adjoint_passes(osbf_ctx *ctx, const float *g, int g_is_output, const uint8_t *maps, int t0, int t1,
                               int P, int H, int W, int r, float *gbuf[2], int *cur, cudaStream_t s) {
    const int FH = H + 2 * r, FW = W + 2 * r, FWp = frame_pitch_f32(FW), MP = maps_pitch(FW);
    const long long mstride = (long long)P * FH * MP;
    if (g_is_output) {
        for (int p0 = 0; p0 < P; p0 += 65535) {
            const int np = P - p0 < 65535 ? P - p0 : 65535;
            dim3 grid((FW + 255) / 256 < 8 ? (FW + 255) / 256 : 8, FH, np);
            embed_zero_kernel<<<grid, 256, 0, s>>>(g + (size_t)p0 * H * W, gbuf[0] + (size_t)p0 * FH * FWp, H, W, r,
                                                   FW, FWp);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
            osbf_ctx_count_launches(ctx, 1);
        }
        *cur = 0;
    }
    const bwd::BLayout L = bwd::make_blayout(r);
    int occ = occupancy_bwd(r);
    if (occ < 1) occ = 1;
    const int shift = (16 - r % 16) % 16;  // tile k starts at column k * TW - shift: boxes start on 16 bytes
    bwd::BwdParams p;
    std::memset(&p, 0, sizeof p);
    p.dst_plane = (long long)FH * FWp;
    p.dst_pitch = FWp;
    p.FH = FH;
    p.FW = FW;
    p.tiles_x = (FW - 1 + shift) / bwd::TW + 1;
    p.tiles_y = (FH + bwd::TH - 1) / bwd::TH;
    const long long ntiles = (long long)p.tiles_x * p.tiles_y * P;
    if (ntiles > 0x7fffffffLL) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "too many tiles");
    p.ntiles = (int)ntiles;
    p.tx_shift = shift;
    p.err = osbf_ctx_err_word(ctx);
    const long long gmax = (long long)occ * osbf_ctx_sms(ctx);
    const int grid = (int)(gmax < ntiles ? gmax : ntiles);
    for (int t = t1 - 1; t >= t0; --t) {
        CUtensorMap gmap, mmap;
        if (!encode_frame_map(&gmap, Storage::F32, gbuf[*cur], FW, FH, P, FWp, L.BXg, L.RH) ||
            !encode_frame_map(&mmap, Storage::U8, maps + t * mstride, FW, FH, P, MP, L.BXm, L.RH))
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "cuTensorMapEncodeTiled failed (backward)");
        const int nxt = 1 - *cur;
        p.gdst = gbuf[nxt];
        cudaError_t e = launch_bwd(r, gmap, mmap, p, grid, s);
        if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
        osbf_ctx_count_launches(ctx, 1);
        *cur = nxt;
    }
    return OSBF_OK;
}

osbf_status fold_pad(osbf_ctx *ctx, const float *gframe, float *grad_in, int P, int H, int W, int r, cudaStream_t s) {
    const int FW = W + 2 * r, FWp = frame_pitch_f32(FW);
    for (int p0 = 0; p0 < P; p0 += 65535) {
        const int np = P - p0 < 65535 ? P - p0 : 65535;
        dim3 grid((W + 255) / 256 < 16 ? (W + 255) / 256 : 16, H, np);
        pad_adjoint_kernel<<<grid, 256, 0, s>>>(gframe + (size_t)p0 * (H + 2 * r) * FWp,
                                                grad_in + (size_t)p0 * H * W, H, W, r, FW, FWp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
        osbf_ctx_count_launches(ctx, 1);
    }
    return OSBF_OK;
}

}  // namespace

osbf_status osbf_backward_impl(osbf_ctx *ctx, const float *grad_out, float *grad_in, const uint8_t *maps, int P, int H,
                               int W, int r, int iters, cudaStream_t s) {
    const int FH = H + 2 * r, FWp = frame_pitch_f32(W + 2 * r);
    const size_t fb = sizeof(float) * (size_t)P * FH * FWp;
    osbf_status st;
    float *gbuf[2];
    gbuf[0] = (float *)osbf_ctx_workspace(ctx, 0, fb, &st);
    if (st) return st;
    gbuf[1] = (float *)osbf_ctx_workspace(ctx, 1, fb, &st);
    if (st) return st;
    int cur = 0;
    st = run_adjoint_passes(ctx, grad_out, 1, maps, 0, iters, P, H, W, r, gbuf, &cur, s);
    if (st) return st;
    return fold_pad(ctx, gbuf[cur], grad_in, P, H, W, r, s);
}

extern "C" {

int osbf_frame_pitch(int W, int r) { return frame_pitch_f32(W + 2 * r); }

int osbf_maps_pitch(int W, int r) { return maps_pitch(W + 2 * r); }

osbf_status osbf_filter_checkpointed(osbf_ctx *ctx, const float *in, float *out, float *checkpoints, int interval,
                                     int N, int C, int H, int W, int r, int iters, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    osbf_ctx_reset_launches(ctx);
    if (!in || !out || (!checkpoints && iters > 0)) return osbf_ctx_fail(ctx, OSBF_EINVAL, "null pointer");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0 || interval <= 0)
        return osbf_ctx_fail(ctx, OSBF_EINVAL, "bad sizes, r, iters or interval");
    if (r > OSBF_MAX_RADIUS) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "r exceeds OSBF_MAX_RADIUS");
    const int P = N * C, FH = H + 2 * r, FW = W + 2 * r, FWp = frame_pitch_f32(FW);
    const long long fstride = (long long)P * FH * FWp;
    cudaStream_t s = (cudaStream_t)stream;
    if (iters == 0 || r == 0) {
        if (cudaMemcpyAsync(out, in, sizeof(float) * (size_t)P * H * W, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "copy failed");
        if (iters > 0) {  // r == 0: the state never changes; every checkpoint is the input frame
            const int K = (iters + interval - 1) / interval;
            for (int k = 0; k < K; ++k) {
                if (launch_pad_replicate(Storage::F32, in, checkpoints + k * fstride, P, H, W, 0, FH, FW, FWp, s) !=
                    cudaSuccess)
                    return osbf_ctx_fail(ctx, OSBF_ECUDA, "pad failed");
            }
        }
        return OSBF_OK;
    }
    const int K = (iters + interval - 1) / interval;
    cudaError_t e = launch_pad_replicate(Storage::F32, in, checkpoints, P, H, W, r, FH, FW, FWp, s);
    if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
    osbf_ctx_count_launches(ctx, 1);
    for (int k = 1; k < K; ++k) {
        osbf_status st = osbf_forward_run(ctx, checkpoints + (k - 1) * fstride, 1, FWp, checkpoints + k * fstride, 1,
                                          FWp, P, H, W, r, interval, OSBF_F32, 0, 0, nullptr, 0, 0, s);
        if (st) return st;
    }
    return osbf_forward_run(ctx, checkpoints + (K - 1) * fstride, 1, FWp, out, 0, 0, P, H, W, r,
                            iters - (K - 1) * interval, OSBF_F32, 0, 0, nullptr, 0, 0, s);
}

osbf_status osbf_filter_backward_checkpointed(osbf_ctx *ctx, const float *grad_out, float *grad_in,
                                              const float *checkpoints, int interval, int N, int C, int H, int W,
                                              int r, int iters, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    osbf_ctx_reset_launches(ctx);
    if (!grad_out || !grad_in || (!checkpoints && iters > 0)) return osbf_ctx_fail(ctx, OSBF_EINVAL, "null pointer");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0 || interval <= 0)
        return osbf_ctx_fail(ctx, OSBF_EINVAL, "bad sizes, r, iters or interval");
    if (r > OSBF_MAX_RADIUS) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "r exceeds OSBF_MAX_RADIUS");
    const int P = N * C, FH = H + 2 * r, FW = W + 2 * r, FWp = frame_pitch_f32(FW);
    cudaStream_t s = (cudaStream_t)stream;
    if (iters == 0 || r == 0) {
        if (cudaMemcpyAsync(grad_in, grad_out, sizeof(float) * (size_t)P * H * W, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "copy failed");
        return OSBF_OK;
    }
    const long long fstride = (long long)P * FH * FWp;
    const long long mstride = (long long)P * FH * maps_pitch(FW);
    const int K = (iters + interval - 1) / interval;
    osbf_status st;
    const size_t fb = sizeof(float) * (size_t)fstride;
    float *gbuf[2];
    gbuf[0] = (float *)osbf_ctx_workspace(ctx, 0, fb, &st);
    if (st) return st;
    gbuf[1] = (float *)osbf_ctx_workspace(ctx, 1, fb, &st);
    if (st) return st;
    uint8_t *wmaps = (uint8_t *)osbf_ctx_workspace(ctx, 2, (size_t)mstride * interval, &st);
    if (st) return st;
    float *scratch = (float *)osbf_ctx_workspace(ctx, 3, fb, &st);
    if (st) return st;
    int cur = 0;
    int first = 1;
    for (int k = K - 1; k >= 0; --k) {
        const int seg = k == K - 1 ? iters - k * interval : interval;
        // recompute this segment's selections from its checkpoint
        st = osbf_forward_run(ctx, checkpoints + k * fstride, 1, FWp, scratch, 1, FWp, P, H, W, r, seg, OSBF_F32, 0, 0,
                              wmaps, 0, mstride, s);
        if (st) return st;
        st = run_adjoint_passes(ctx, grad_out, first, wmaps, 0, seg, P, H, W, r, gbuf, &cur, s);
        if (st) return st;
        first = 0;
    }
    return fold_pad(ctx, gbuf[cur], grad_in, P, H, W, r, s);
}

}  // extern "C"
