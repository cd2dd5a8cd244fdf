// Backward of the One-Sided Box Filter: per-pass adjoint launches (osbf_bwd.cuh), the
// transpose of the appendix's replicate padding, and the checkpointed forward/backward.
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

static cudaError_t launch_bwd(int R, const bwd::BwdParams &p, dim3 grid, cudaStream_t s) {
    switch (R) {
#define OSBF_CASE(RR) \
    case RR: return bwd::launch_bwd_tile<RR>(p, grid, s);
        OSBF_FOR_EACH_R(OSBF_CASE)
#undef OSBF_CASE
    }
    return cudaErrorInvalidValue;
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

namespace {

int frame_pitch_f32(int FW) { return (FW + 31) / 32 * 32; }

// The backward passes t = t1-1 .. t0 (maps + t * stride), starting from `g` (the caller's
// grad_out when g_is_output, else a gradient frame); the result lands in one of two
// gradient frames, returned through *result.
osbf_status run_adjoint_passes(osbf_ctx *ctx, const float *g, int g_is_output, const uint8_t *maps, int t0, int t1,
                               int P, int H, int W, int r, float *gbuf[2], int *cur, cudaStream_t s) {
    const int FH = H + 2 * r, FW = W + 2 * r, FWp = frame_pitch_f32(FW);
    const long long mstride = (long long)P * FH * FW;
    for (int t = t1 - 1; t >= t0; --t) {
        bwd::BwdParams p;
        std::memset(&p, 0, sizeof p);
        if (g_is_output) {
            p.gsrc = g;
            p.src_is_output = 1;
            p.src_plane = (long long)H * W;
            p.src_pitch = W;
        } else {
            p.gsrc = gbuf[*cur];
            p.src_plane = (long long)FH * FWp;
            p.src_pitch = FWp;
        }
        const int nxt = g_is_output ? 0 : 1 - *cur;
        p.gdst = gbuf[nxt];
        p.dst_plane = (long long)FH * FWp;
        p.dst_pitch = FWp;
        p.maps = maps + (long long)t * mstride;
        p.H = H;
        p.W = W;
        p.FH = FH;
        p.FW = FW;
        p.R = r;
        for (int p0 = 0; p0 < P; p0 += 65535) {
            const int np = P - p0 < 65535 ? P - p0 : 65535;
            bwd::BwdParams q = p;
            q.gsrc = p.gsrc + (size_t)p0 * p.src_plane;
            q.gdst = p.gdst + (size_t)p0 * p.dst_plane;
            q.maps = p.maps + (size_t)p0 * FH * FW;
            dim3 grid((FW + bwd::TW - 1) / bwd::TW, (FH + bwd::TH - 1) / bwd::TH, np);
            cudaError_t e = launch_bwd(r, q, grid, s);
            if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
            osbf_ctx_count_launches(ctx, 1);
        }
        *cur = nxt;
        g_is_output = 0;
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
    const long long mstride = (long long)P * FH * FW;
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
