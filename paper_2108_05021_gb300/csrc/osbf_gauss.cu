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
// Separable sums, one CTA per TH x TW tile of a frame, its region (TH + 2r) x 128 by one
// TMA box:
//   pass V (thread = column pair x 8 output rows, packed f32x2 over the pair):
//     Up(y) = sum_k wh[k] V(y-k),  Dn(y) = sum_k wh[k] V(y+k),
//     Fy(y) = c (Up + Dn) - wf0 V(y)           (c = wf[k] / wh[k]: the full column mean is
//                                               the two halves with the centre taken once);
//   pass H (thread = 8 consecutive outputs of one row): left / right sums
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

// NT threads; TH output rows per tile (4 pass-V segments of SEG rows); every tile region
// is RW = 128 columns wide, its TW = RW - 2 RP output columns centred (RP = r rounded up to
// a multiple of 4, so region and output columns both start on 16 bytes); G outputs per
// pass-H thread.
constexpr int NT = 256, TH = 32, SEG = 8, RW = 128, G = 8;
static_assert(TH == SEG * (NT / (RW / 2)), "pass V: one thread per column pair and segment");

__host__ __device__ constexpr int rp(int R) { return (R + 3) / 4 * 4; }
__host__ __device__ constexpr int r2(int R) { return (R + 1) / 2 * 2; }
__host__ __device__ constexpr int tw(int R) { return RW - 2 * rp(R); }
__host__ __device__ constexpr int rh(int R) { return TH + 2 * R; }
// shared layout (bytes): the region V (RH x RW floats, as the TMA box lands), the {Up, Dn}
// pairs (TH x RW float2, 16-byte chunks swizzled), Fy (TH x RW floats, chunks swizzled), the
// mbarrier
__host__ __device__ constexpr int off_ud(int R) { return rh(R) * RW * 4; }
__host__ __device__ constexpr int off_f(int R) { return off_ud(R) + TH * RW * 8; }
__host__ __device__ constexpr int smem_bytes(int R) { return off_f(R) + TH * RW * 4 + 16; }

// The chunk swizzles keep pass H's strided 16-byte loads (lane stride G/2 chunks of
// {Up, Dn}, G/4 chunks of Fy) on distinct banks within each 8-lane phase.
__device__ __forceinline__ int ud_chunk(int q) { return q ^ ((q >> 3) & 3); }
__device__ __forceinline__ int f_chunk(int q) { return q ^ ((q >> 3) & 1); }

struct GaussParams {
    float wh[OSBF_MAX_RADIUS_GAUSS + 1];  // one-sided weights, distance 0..r
    float c, wf0;                         // wf[k] / wh[k] and wf[0]
    float *dst;                           // next frame: P x FH x FWp
    uint8_t *maps;                        // this pass's maps (P x FH x map_pitch) or null
    long long dst_plane, map_plane;
    int map_pitch, FH, FW, FWp, tiles_x;
    unsigned int *err;                    // bit 0: a tile load did not land in time
};

__device__ __forceinline__ float2 bc(float w) { return make_float2(w, w); }

// pass V: thread = column pair cp and a segment of SEG output rows; region rows
// seg*SEG + j, j = 0..SEG+2R-1, enter one at a time; output row i of the segment is region
// row i + R.
template <int R>
__device__ __forceinline__ void pass_v(const float *bV, float4 *ud, float4 *fy, const GaussParams &q) {
    const int cp = threadIdx.x & (RW / 2 - 1), seg = threadIdx.x / (RW / 2);
    const float2 *src = reinterpret_cast<const float2 *>(bV) + seg * SEG * (RW / 2) + cp;
    const float2 c2 = bc(q.c), m2 = bc(-q.wf0);
    float2 up[SEG], dn[SEG], fc[SEG];
#pragma unroll
    for (int j = 0; j < SEG + 2 * R; ++j) {
        const float2 v = src[j * (RW / 2)];
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            const int kl = i + R - j, kr = j - i - R;  // tap distance for Up(i) / Dn(i)
            if (kl >= 0 && kl <= R) up[i] = kl == R ? v2::mul2(bc(q.wh[kl]), v) : v2::fma2(bc(q.wh[kl]), v, up[i]);
            if (kr >= 0 && kr <= R) dn[i] = kr == 0 ? v2::mul2(bc(q.wh[kr]), v) : v2::fma2(bc(q.wh[kr]), v, dn[i]);
            if (kr == 0) fc[i] = v2::mul2(m2, v);
            if (kr == R) {  // row i complete
                const float2 f = v2::fma2(c2, v2::add2(up[i], dn[i]), fc[i]);
                const int o = seg * SEG + i;
                ud[o * (RW / 2) + ud_chunk(cp)] = make_float4(up[i].x, dn[i].x, up[i].y, dn[i].y);
                reinterpret_cast<float2 *>(fy + o * (RW / 4) + f_chunk(cp >> 1))[cp & 1] = f;
            }
        }
    }
}

// pass H: thread = G consecutive outputs (region columns c0..c0+G-1) of one output row.
template <int R>
__device__ __forceinline__ void pass_h(const float *bV, const float4 *ud, const float4 *fy, const GaussParams &q,
                                       int plane, int ty0, int tx0) {
    constexpr int RP = rp(R), R2 = r2(R), TW = tw(R), NG = TW / G;
    constexpr int NUD = (G + 2 * R2) / 2;  // chunks of {Up, Dn} pairs, from column c0 - R2
    constexpr int NF = (G + 2 * RP) / 4;   // chunks of Fy, from column c0 - RP
    static_assert(TW % G == 0 && G % 4 == 0, "output groups of whole 16-byte chunks");
    const float2 c2 = bc(q.c), m2 = bc(-q.wf0);
    for (int it = threadIdx.x; it < TH * NG; it += NT) {
        const int row = it / NG, g = it - row * NG;
        const int c0 = RP + G * g;
        float u[G];
#pragma unroll
        for (int h = 0; h < G / 4; ++h) {
            const float4 t = reinterpret_cast<const float4 *>(bV + (row + R) * RW + c0)[h];
            u[4 * h] = t.x;
            u[4 * h + 1] = t.y;
            u[4 * h + 2] = t.z;
            u[4 * h + 3] = t.w;
        }
        // {Up, Dn}: left and right sums, the centre pair for the full-row means
        float2 lt[G], rt[G], xc[G];
        const float4 *udr = ud + row * (RW / 2);
        const int q0 = (c0 - R2) >> 1;
#pragma unroll
        for (int m = 0; m < NUD; ++m) {
            const float4 t = udr[ud_chunk(q0 + m)];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 v = h ? make_float2(t.z, t.w) : make_float2(t.x, t.y);
                const int p = 2 * m + h;  // column c0 - R2 + p
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int kl = o + R2 - p, kr = p - R2 - o;
                    if (kl >= 0 && kl <= R)
                        lt[o] = kl == R ? v2::mul2(bc(q.wh[kl]), v) : v2::fma2(bc(q.wh[kl]), v, lt[o]);
                    if (kr >= 0 && kr <= R)
                        rt[o] = kr == 0 ? v2::mul2(bc(q.wh[kr]), v) : v2::fma2(bc(q.wh[kr]), v, rt[o]);
                    if (kr == 0) xc[o] = v2::mul2(m2, v);
                }
            }
        }
        // candidates N1..N4 (best A) and N7, N8 (best B), first argmin within each group
        float bA[G], aA[G], bB[G], aB[G];
        int iA[G], iB[G];
#pragma unroll
        for (int o = 0; o < G; ++o) {
            const float2 f = v2::fma2(c2, v2::add2(lt[o], rt[o]), xc[o]);  // {N8, N7}
            const float m1 = lt[o].y, mm2 = rt[o].y, m3 = rt[o].x, m4 = lt[o].x;
            float b = m1, a = fabsf(m1 - u[o]);
            int i = 1;
            float t = fabsf(mm2 - u[o]);
            if (t < a) { b = mm2; a = t; i = 2; }
            t = fabsf(m3 - u[o]);
            if (t < a) { b = m3; a = t; i = 3; }
            t = fabsf(m4 - u[o]);
            if (t < a) { b = m4; a = t; i = 4; }
            bA[o] = b;
            aA[o] = a;
            iA[o] = i;
            const float a7 = fabsf(f.y - u[o]), a8 = fabsf(f.x - u[o]);
            const bool p8 = a8 < a7;
            bB[o] = p8 ? f.x : f.y;
            aB[o] = p8 ? a8 : a7;
            iB[o] = p8 ? 8 : 7;
        }
        // Fy: left and right sums (N5, N6)
        float lf[G], rf[G];
        const float4 *fr = fy + row * (RW / 4);
        const int f0 = (c0 - RP) >> 2;
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            const float4 t = fr[f_chunk(f0 + m)];
            const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int p = 4 * m + h;  // column c0 - RP + p
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    const int kl = o + RP - p, kr = p - RP - o;
                    if (kl >= 0 && kl <= R) lf[o] = kl == R ? q.wh[kl] * tv[h] : fmaf(q.wh[kl], tv[h], lf[o]);
                    if (kr >= 0 && kr <= R) rf[o] = kr == 0 ? q.wh[kr] * tv[h] : fmaf(q.wh[kr], tv[h], rf[o]);
                }
            }
        }
        float res[G];
        uint8_t sel[G];
#pragma unroll
        for (int o = 0; o < G; ++o) {  // order: N1..N4, N5, N6, N7..N8
            float b = bA[o], a = aA[o];
            int i = iA[o];
            float t = fabsf(lf[o] - u[o]);
            if (t < a) { b = lf[o]; a = t; i = 5; }
            t = fabsf(rf[o] - u[o]);
            if (t < a) { b = rf[o]; a = t; i = 6; }
            if (aB[o] < a) { b = bB[o]; i = iB[o]; }
            res[o] = b;
            sel[o] = (uint8_t)i;
        }
        const int y = ty0 + row, x = tx0 + G * g;
        if (y < q.FH && x < q.FW) {
            float *d = q.dst + (long long)plane * q.dst_plane + (long long)y * q.FWp + x;
#pragma unroll
            for (int h = 0; h < G / 4; ++h)  // rows are padded to 4 floats: a started 4-vector fits
                if (x + 4 * h < q.FW)
                    reinterpret_cast<float4 *>(d)[h] = make_float4(res[4 * h], res[4 * h + 1], res[4 * h + 2], res[4 * h + 3]);
            if (q.maps) {
                uint8_t *mp = q.maps + (long long)plane * q.map_plane + (long long)y * q.map_pitch + x;
                uint32_t w[G / 4];
#pragma unroll
                for (int h = 0; h < G / 4; ++h)
                    w[h] = sel[4 * h] | (sel[4 * h + 1] << 8) | (sel[4 * h + 2] << 16) | ((uint32_t)sel[4 * h + 3] << 24);
#pragma unroll
                for (int h = 0; h < G / 4; ++h)  // map rows are padded to 16 bytes
                    if (x + 4 * h < q.FW) reinterpret_cast<uint32_t *>(mp)[h] = w[h];
            }
        }
    }
}

template <int R>
__global__ void __launch_bounds__(NT, 3) gauss_kernel(const __grid_constant__ CUtensorMap src, const GaussParams q) {
    extern __shared__ __align__(128) unsigned char smg[];
    float *bV = reinterpret_cast<float *>(smg);
    float4 *ud = reinterpret_cast<float4 *>(smg + off_ud(R));
    float4 *fy = reinterpret_cast<float4 *>(smg + off_f(R));
    const uint32_t bar = v2::smem_u32(smg + smem_bytes(R) - 16);
    const int tile = blockIdx.x, plane = blockIdx.y;
    const int ty0 = (tile / q.tiles_x) * TH, tx0 = (tile % q.tiles_x) * tw(R);
    if (threadIdx.x == 0) {
        v2::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        v2::fence_proxy_async();
        v2::tma_load_3d(v2::smem_u32(bV), &src, tx0 - rp(R), ty0 - R, plane, bar, (uint32_t)(rh(R) * RW * 4));
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
    pass_h<R>(bV, ud, fy, q, plane, ty0, tx0);
}

template <int R>
cudaError_t launch(const CUtensorMap &m, const GaussParams &q, int tiles, int P, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gauss_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(R));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gauss_kernel<R><<<dim3(tiles, P), NT, smem_bytes(R), s>>>(m, q);
    return cudaGetLastError();
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
        for (int k = 0; k <= r; ++k) q.wh[k] = (float)(g[k] / sh);
        q.c = (float)(sh / sf);
        q.wf0 = (float)(g[0] / sf);
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
        if (!encode_frame_map(&m, Storage::F32, fr[cur], FW, FH, (int)P, FWp, vg::RW, vg::region_rows(r)))
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
