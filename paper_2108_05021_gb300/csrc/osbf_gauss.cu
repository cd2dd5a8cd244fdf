// The one-sided Gaussian filter: Algorithm 1 with Phi = a weighted mean whose kernels are
// built as in Sec. "Separable Kernels" from the Gaussian k(u) = exp(-u^2 / (2 sigma^2)),
// u = -r..r.  Per axis two normalised 1D kernels: the one-sided wh[k] = k(k) / sum_{0..r} k
// (distance k = 0..r from the centre, centre included on both sides) and the full
// wf[k] = k(k) / sum_{-r..r} k.  Window N_i's 2D kernel is the product of one 1D kernel
// per axis: one-sided on an axis the window halves, full on an axis it spans (quadrants
// N1..N4: one-sided x one-sided; N5, N6: one-sided in x, full in y; N7, N8: full in x,
// one-sided in y).  Selection and update as Algorithm 2 (first argmin |mean - U| in the
// order N1..N8); the appendix's boundary (replicate pad by r once, zeros outside the
// frame, not renormalised there, crop at the end).
//
// Separable sums, one CTA per TH x TW tile of a frame, its region (TH + 2r) x 120 by one
// TMA box:
//   pass V (thread = column pair x 8 output rows, packed f32x2 over the pair):
//     Up(y) = sum_k wh[k] V(y-k),  Dn(y) = sum_k wh[k] V(y+k),
//     Fy(y) = c (Up + Dn) - wf0 V(y)           (c = wf[k] / wh[k]: the full column mean is
//                                               the two halves with the centre taken once);
//   pass H (lane = row, thread = 8 consecutive outputs of its row): left / right sums
//     L(X)(x) = sum_k wh[k] X(x-k), Rt(X)(x) = sum_k wh[k] X(x+k) of the pair {Up, Dn}
//     (packed) and of Fy, then
//       N1 = L(Dn), N2 = Rt(Dn), N3 = Rt(Up), N4 = L(Up), N5 = L(Fy), N6 = Rt(Fy),
//       N7 = c (L(Dn) + Rt(Dn)) - wf0 Dn(x),  N8 = c (L(Up) + Rt(Up)) - wf0 Up(x).
// Every weighted sum is formed afresh from its taps (no running sums).
#include <cmath>
#include <cstring>

#include "osbf.h"
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg);
void *osbf_ctx_workspace(osbf_ctx *ctx, int slot, size_t bytes, osbf_status *st);
void osbf_ctx_count_launches(osbf_ctx *ctx, int n);
void osbf_ctx_reset_launches(osbf_ctx *ctx);
unsigned int *osbf_ctx_err_word(osbf_ctx *ctx);

namespace osbf {
namespace vg {

// NT threads; TH output rows per tile (4 pass-V segments of SEG rows; in pass H lane = row);
// every tile region is RW = 120 columns wide, its TW = RW - 2 RP output columns centred (RP
// = r rounded up to a multiple of 4, so region and output columns both start on 16 bytes);
// G outputs per pass-H thread.
constexpr int NT = 256, TH = 32, SEG = 8, RW = 120, G = 8;
static_assert(TH == 32 && TH == SEG * (NT / 64), "pass V: column pair x segment; pass H: lane = row");
// Row pitches (floats) of the shared fields, odd numbers of 16-byte chunks: the lane = row
// 16-byte loads of pass H fall on distinct banks in every 8-lane phase.  VP is also the
// TMA box width (4 columns past the region, unused).
constexpr int VP = RW + 4, UDP = 2 * RW + 4, FP = RW + 4;
static_assert((VP / 4) % 2 == 1 && (UDP / 4) % 2 == 1 && (FP / 4) % 2 == 1, "odd chunk pitches");

__host__ __device__ constexpr int rp(int R) { return (R + 3) / 4 * 4; }
__host__ __device__ constexpr int r2(int R) { return (R + 1) / 2 * 2; }
__host__ __device__ constexpr int tw(int R) { return RW - 2 * rp(R); }
__host__ __device__ constexpr int rh(int R) { return TH + 2 * R; }
// shared layout (bytes): the region V (RH rows of VP floats, as the TMA box lands), the
// {Up, Dn} pairs (TH rows of UDP floats), Fy (TH rows of FP floats), the mbarrier
__host__ __device__ constexpr int off_ud(int R) { return rh(R) * VP * 4; }
__host__ __device__ constexpr int off_f(int R) { return off_ud(R) + TH * UDP * 4; }
__host__ __device__ constexpr int smem_bytes(int R) { return off_f(R) + TH * FP * 4 + 16; }

struct GaussParams {
    float2 wh2[OSBF_MAX_RADIUS_GAUSS + 1];  // {wh[k], wh[k]}: one-sided weights, distance 0..r
    float wh[OSBF_MAX_RADIUS_GAUSS + 1];
    float2 c2, m2;                          // {wf[k] / wh[k]} and {-wf[0]}, pairs
    float *dst;                             // next frame: P x FH x FWp
    uint8_t *maps;                          // this pass's maps (P x FH x map_pitch) or null
    long long dst_plane, map_plane;
    int map_pitch, FH, FW, FWp, tiles_x;
    unsigned int *err;                      // bit 0: a tile load did not land in time
};

// pass V: thread = column pair cp (< RW/2) and a segment of SEG output rows; region rows
// seg*SEG + j, j = 0..SEG+2R-1, enter one at a time; output row i of the segment is region
// row i + R.
template <int R>
__device__ __forceinline__ void pass_v(const float *bV, float *ud, float *fy, const GaussParams &q) {
    const int cp = threadIdx.x & 63, seg = threadIdx.x >> 6;
    if (cp >= RW / 2) return;
    const float *src = bV + seg * SEG * VP + 2 * cp;
    const float2 c2 = q.c2, m2 = q.m2;
    float2 up[SEG], dn[SEG], fc[SEG];
#pragma unroll
    for (int j = 0; j < SEG + 2 * R; ++j) {
        const float2 v = *reinterpret_cast<const float2 *>(src + j * VP);
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            const int kl = i + R - j, kr = j - i - R;  // tap distance for Up(i) / Dn(i)
            if (kl >= 0 && kl <= R) up[i] = kl == R ? v2::mul2(q.wh2[kl], v) : v2::fma2(q.wh2[kl], v, up[i]);
            if (kr >= 0 && kr <= R) dn[i] = kr == 0 ? v2::mul2(q.wh2[kr], v) : v2::fma2(q.wh2[kr], v, dn[i]);
            if (kr == 0) fc[i] = v2::mul2(m2, v);
            if (kr == R) {  // row i complete
                const float2 f = v2::fma2(c2, v2::add2(up[i], dn[i]), fc[i]);
                const int o = seg * SEG + i;
                *reinterpret_cast<float4 *>(ud + o * UDP + 4 * cp) = make_float4(up[i].x, dn[i].x, up[i].y, dn[i].y);
                *reinterpret_cast<float2 *>(fy + o * FP + 2 * cp) = f;
            }
        }
    }
}

// pass H: lane = output row, warp = a group of G consecutive output columns (region columns
// c0..c0+G-1).  Selection by signed differences d_i = mean_i - U, first argmin |d_i| in
// the order N1..N8, U <- U + d (Algorithm 2).  Evaluated in that order as three groups:
// once both sums of an output are complete, the best of N1..N4 and, kept apart, the best
// of N7, N8; after the Fy sums, N5 and N6 against the first, then the N7 / N8 winner -- a
// later window replaces the best only when strictly closer.
template <int R, bool MAPS>
__device__ __forceinline__ void pass_h(const float *bV, const float *ud, const float *fy, const GaussParams &q,
                                       int plane, int ty0, int tx0) {
    constexpr int RP = rp(R), R2 = r2(R), TW = tw(R), NG = TW / G;
    constexpr int NUD = (G + 2 * R2) / 2;  // 16-byte chunks of {Up, Dn} pairs, from column c0 - R2
    constexpr int NF = (G + 2 * RP) / 4;   // 16-byte chunks of Fy, from column c0 - RP
    static_assert(TW % G == 0 && G % 4 == 0, "output groups of whole 16-byte chunks");
    const int row = threadIdx.x & 31;
    const float2 c2 = q.c2, m2 = q.m2;
    for (int g = threadIdx.x >> 5; g < NG; g += NT / 32) {
        const int c0 = RP + G * g;
        const float *urow = bV + (row + R) * VP + c0;  // the outputs' own values U, read where used
        float bd[G], bb[G];   // best signed difference of N1..N4 / of N7, N8
        int bi[G];            // MAPS: their windows (low / high nibble), then the chosen one
        float2 lt[G], rt[G], xc[G];
        const float4 *udr = reinterpret_cast<const float4 *>(ud + row * UDP + 2 * (c0 - R2));
#pragma unroll
        for (int m = 0; m < NUD; ++m) {
            const float4 t = udr[m];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 v = h ? make_float2(t.z, t.w) : make_float2(t.x, t.y);
                const int p = 2 * m + h;  // column c0 - R2 + p
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int kl = o + R2 - p, kr = p - R2 - o;
                    if (kl >= 0 && kl <= R) lt[o] = kl == R ? v2::mul2(q.wh2[kl], v) : v2::fma2(q.wh2[kl], v, lt[o]);
                    if (kr >= 0 && kr <= R) rt[o] = kr == 0 ? v2::mul2(q.wh2[kr], v) : v2::fma2(q.wh2[kr], v, rt[o]);
                    if (kr == 0) xc[o] = v2::mul2(m2, v);
                    if (kr == R) {  // both sums of output o complete: N1..N4, N7, N8
                        const float2 f = v2::fma2(c2, v2::add2(lt[o], rt[o]), xc[o]);  // {N8, N7}
                        const float uo = urow[o];
                        float d = lt[o].y - uo;
                        int i = 1;
                        float t2 = rt[o].y - uo;
                        if (fabsf(t2) < fabsf(d)) { d = t2; i = 2; }
                        t2 = rt[o].x - uo;
                        if (fabsf(t2) < fabsf(d)) { d = t2; i = 3; }
                        t2 = lt[o].x - uo;
                        if (fabsf(t2) < fabsf(d)) { d = t2; i = 4; }
                        float db = f.y - uo;
                        int ib = 7;
                        t2 = f.x - uo;
                        if (fabsf(t2) < fabsf(db)) { db = t2; ib = 8; }
                        bd[o] = d;
                        bb[o] = db;
                        if (MAPS) bi[o] = i | (ib << 4);
                    }
                }
            }
        }
        // Fy: left and right sums (N5, N6)
        float lf[G], rf[G];
        const float4 *fr = reinterpret_cast<const float4 *>(fy + row * FP + (c0 - RP));
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            const float4 t = fr[m];
            const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int p = 4 * m + h;  // column c0 - RP + p
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int kl = o + RP - p, kr = p - RP - o;
                    if (kl >= 0 && kl <= R) lf[o] = kl == R ? q.wh[kl] * tv[h] : fmaf(q.wh[kl], tv[h], lf[o]);
                    if (kr >= 0 && kr <= R) rf[o] = kr == 0 ? q.wh[kr] * tv[h] : fmaf(q.wh[kr], tv[h], rf[o]);
                    if (kr == R) {
                        float d = bd[o];
                        int i = MAPS ? bi[o] & 15 : 0;
                        const float uo = urow[o];
                        const float d5 = lf[o] - uo, d6 = rf[o] - uo;
                        if (fabsf(d5) < fabsf(d)) { d = d5; i = 5; }
                        if (fabsf(d6) < fabsf(d)) { d = d6; i = 6; }
                        if (fabsf(bb[o]) < fabsf(d)) { d = bb[o]; i = MAPS ? bi[o] >> 4 : 0; }
                        bd[o] = uo + d;  // the updated value
                        if (MAPS) bi[o] = i;
                    }
                }
            }
        }
        const int y = ty0 + row, x = tx0 + G * g;
        if (y < q.FH && x < q.FW) {
            float *dp = q.dst + (long long)plane * q.dst_plane + (long long)y * q.FWp + x;
#pragma unroll
            for (int h = 0; h < G / 4; ++h)  // rows are padded to 4 floats: a started 4-vector fits
                if (x + 4 * h < q.FW)
                    reinterpret_cast<float4 *>(dp)[h] = make_float4(bd[4 * h], bd[4 * h + 1], bd[4 * h + 2], bd[4 * h + 3]);
            if (MAPS) {
                uint8_t *mp = q.maps + (long long)plane * q.map_plane + (long long)y * q.map_pitch + x;
#pragma unroll
                for (int h = 0; h < G / 4; ++h)  // map rows are padded to 16 bytes
                    if (x + 4 * h < q.FW)
                        reinterpret_cast<uint32_t *>(mp)[h] = (uint32_t)bi[4 * h] | ((uint32_t)bi[4 * h + 1] << 8) |
                                                              ((uint32_t)bi[4 * h + 2] << 16) |
                                                              ((uint32_t)bi[4 * h + 3] << 24);
            }
        }
    }
}

// CTAs per SM the shared layout allows (228 KB per SM, 1 KB reserved per CTA)
__host__ __device__ constexpr int ctas_per_sm(int R) { return 228 * 1024 / (smem_bytes(R) + 1024); }

template <int R, bool MAPS>
__global__ void __launch_bounds__(NT, ctas_per_sm(R) >= 3 ? 3 : 2) gauss_kernel(const __grid_constant__ CUtensorMap src, const GaussParams q) {
    extern __shared__ __align__(128) unsigned char smg[];
    float *bV = reinterpret_cast<float *>(smg);
    float *ud = reinterpret_cast<float *>(smg + off_ud(R));
    float *fy = reinterpret_cast<float *>(smg + off_f(R));
    const uint32_t bar = v2::smem_u32(smg + smem_bytes(R) - 16);
    const int tile = blockIdx.x, plane = blockIdx.y;
    const int ty0 = (tile / q.tiles_x) * TH, tx0 = (tile % q.tiles_x) * tw(R);
    if (threadIdx.x == 0) {
        v2::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        v2::fence_proxy_async();
        v2::tma_load_3d(v2::smem_u32(bV), &src, tx0 - rp(R), ty0 - R, plane, bar, (uint32_t)(rh(R) * VP * 4));
    }
    __syncthreads();
    const bool timed_out = !v2::mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(timed_out)) {
        if (threadIdx.x == 0) {
            atomicOr(q.err, 1u);
            v2::mbar_wait_bounded(bar, 0);  // let a late copy land before the CTA leaves
        }
        return;
    }
    pass_v<R>(bV, ud, fy, q);
    __syncthreads();
    pass_h<R, MAPS>(bV, ud, fy, q, plane, ty0, tx0);
}

template <int R, bool MAPS>
cudaError_t launch_m(const CUtensorMap &m, const GaussParams &q, int tiles, int P, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(gauss_kernel<R, MAPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(R));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gauss_kernel<R, MAPS><<<dim3(tiles, P), NT, smem_bytes(R), s>>>(m, q);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch(const CUtensorMap &m, const GaussParams &q, int tiles, int P, cudaStream_t s) {
    return q.maps ? launch_m<R, true>(m, q, tiles, P, s) : launch_m<R, false>(m, q, tiles, P, s);
}

cudaError_t launch_r(int r, const CUtensorMap &m, const GaussParams &q, int tiles, int P, cudaStream_t s) {
    switch (r) {
#define OSBF_GAUSS_CASE(R) \
    case R: return launch<R>(m, q, tiles, P, s);
        OSBF_GAUSS_CASE(1) OSBF_GAUSS_CASE(2) OSBF_GAUSS_CASE(3) OSBF_GAUSS_CASE(4)
        OSBF_GAUSS_CASE(5) OSBF_GAUSS_CASE(6) OSBF_GAUSS_CASE(7) OSBF_GAUSS_CASE(8)
        OSBF_GAUSS_CASE(9) OSBF_GAUSS_CASE(10) OSBF_GAUSS_CASE(11) OSBF_GAUSS_CASE(12)
        OSBF_GAUSS_CASE(13) OSBF_GAUSS_CASE(14) OSBF_GAUSS_CASE(15) OSBF_GAUSS_CASE(16)
#undef OSBF_GAUSS_CASE
    }
    return cudaErrorInvalidValue;
}

int region_rows(int r) { return rh(r); }
int tile_width(int r) { return tw(r); }

}  // namespace vg
}  // namespace osbf

using namespace osbf;

extern "C" osbf_status osbf_filter_gauss(osbf_ctx *ctx, const float *in, float *out, int N, int C, int H, int W,
                                         int r, double sigma, int iters, uint8_t *maps, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    osbf_ctx_reset_launches(ctx);
    if (!in || !out) return osbf_ctx_fail(ctx, OSBF_EINVAL, "null pointer");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0)
        return osbf_ctx_fail(ctx, OSBF_EINVAL, "N, C, H, W must be positive; r, iters >= 0");
    if (!(sigma > 0)) return osbf_ctx_fail(ctx, OSBF_EINVAL, "sigma must be > 0 (+inf: flat weights)");
    if (r > OSBF_MAX_RADIUS_GAUSS) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "r exceeds OSBF_MAX_RADIUS_GAUSS");
    if (maps && ((uintptr_t)maps & 15)) return osbf_ctx_fail(ctx, OSBF_EINVAL, "maps must be 16-byte aligned");
    const long long P = (long long)N * C;
    if (P > 65535) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "N*C exceeds 65535");
    const size_t bytes = sizeof(float) * (size_t)P * H * W;
    if ((const char *)in < (const char *)out + bytes && (const char *)out < (const char *)in + bytes)
        return osbf_ctx_fail(ctx, OSBF_EINVAL, "in and out overlap");
    const int FH = H + 2 * r, FW = W + 2 * r, FWp = (FW + 31) / 32 * 32, MP = maps_pitch(FW);
    const long long mstride = P * FH * MP;
    if (maps && iters > 0) {
        const char *m0 = (const char *)maps, *m1 = m0 + (size_t)mstride * iters;
        if ((m0 < (const char *)in + bytes && (const char *)in < m1) ||
            (m0 < (const char *)out + bytes && (const char *)out < m1))
            return osbf_ctx_fail(ctx, OSBF_EINVAL, "maps overlap an image");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0 || iters == 0) {
        if (cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "copy failed");
        osbf_ctx_count_launches(ctx, 1);
        if (maps && iters > 0) {  // every window is the pixel: N1, first in the order
            if (launch_fill_u8(maps, 1, mstride * iters, s) != cudaSuccess)
                return osbf_ctx_fail(ctx, OSBF_ECUDA, "fill failed");
            osbf_ctx_count_launches(ctx, 1);
        }
        return OSBF_OK;
    }
    vg::GaussParams q;
    std::memset(&q, 0, sizeof q);
    {  // the 1D kernels, in double, rounded once
        double g[OSBF_MAX_RADIUS_GAUSS + 1], sh = 0.0, sf = 0.0;
        for (int k = 0; k <= r; ++k) {
            g[k] = std::exp(-(double)k * k / (2.0 * sigma * sigma));
            sh += g[k];
            sf += k == 0 ? g[k] : 2.0 * g[k];
        }
        for (int k = 0; k <= r; ++k) {
            q.wh[k] = (float)(g[k] / sh);
            q.wh2[k] = make_float2(q.wh[k], q.wh[k]);
        }
        q.c2 = make_float2((float)(sh / sf), (float)(sh / sf));
        q.m2 = make_float2((float)(-g[0] / sf), (float)(-g[0] / sf));
    }
    const size_t fbytes = sizeof(float) * (size_t)P * FH * FWp;
    osbf_status st;
    float *fr[2];
    for (int k = 0; k < 2; ++k) {
        fr[k] = (float *)osbf_ctx_workspace(ctx, k, fbytes, &st);
        if (st) return st;
    }
    cudaError_t e = launch_pad_replicate(Storage::F32, in, fr[0], (int)P, H, W, r, FH, FW, FWp, s);
    if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, "pad launch failed");
    osbf_ctx_count_launches(ctx, 1);
    q.FH = FH;
    q.FW = FW;
    q.FWp = FWp;
    q.dst_plane = (long long)FH * FWp;
    q.map_pitch = MP;
    q.map_plane = (long long)FH * MP;
    q.tiles_x = (FW + vg::tile_width(r) - 1) / vg::tile_width(r);
    q.err = osbf_ctx_err_word(ctx);
    const int tiles = q.tiles_x * ((FH + vg::TH - 1) / vg::TH);
    int cur = 0;
    for (int pass = 0; pass < iters; ++pass) {
        CUtensorMap m;
        if (!encode_frame_map(&m, Storage::F32, fr[cur], FW, FH, (int)P, FWp, vg::VP, vg::region_rows(r)))
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "cuTensorMapEncodeTiled failed (Gaussian frame)");
        q.dst = fr[1 - cur];
        q.maps = maps ? maps + (long long)pass * mstride : nullptr;
        e = vg::launch_r(r, m, q, tiles, (int)P, s);
        if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
        osbf_ctx_count_launches(ctx, 1);
        cur = 1 - cur;
    }
    e = launch_crop_f32(fr[cur], out, (int)P, H, W, r, FWp, s);
    if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, "crop launch failed");
    osbf_ctx_count_launches(ctx, 1);
    return OSBF_OK;
}
