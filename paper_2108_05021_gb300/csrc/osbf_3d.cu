// The 3D one-sided box filter (Sec. "Higher Dimension Case"): eight octant windows of
// (r+1)^3 voxels and six half windows of (r+1)(2r+1)^2 voxels, the selection and update of
// Algorithm 2, the appendix's boundary extended to volumes (replicate pad by r on every
// axis once, zeros beyond the padded volume, crop at the end).  Window order (= tie
// order): O1..O4 = depth z-r..z with the 2D quadrants N1..N4 in (y, x), O5..O8 = depth
// z..z+r with N1..N4, H9 = x-r..x, H10 = x..x+r, H11 = y..y+r, H12 = y-r..y (full on the
// other two axes), H13 = z-r..z, H14 = z..z+r (full in x and y).
//
// Separable sums, per pass:
//   z-pass   (one thread per (y, x) column, register ring over 2r+1 depths):
//            Zm(z) = sum_{z-r..z} U,  Zp(z) = sum_{z..z+r} U  (two fields, frame layout);
//   yx-pass  (per depth slice, 32 x 64 tiles): pass V keeps up-column sums of Zm, Zp and U
//            (Y-(X)(y) = sum_{y-r..y} X; Y+(X)(y) = Y-(X)(y+r)); pass H (lane = row) forms
//            nine row fields from them and slides their left sums L(x) = sum_{x-r..x}:
//              octant (z-, y+/-, x-/+) = L(Y+/-(Zm))(x or x+r), likewise with Zp for z+;
//              H9 / H10 = L(Yf(Zf))(x) / (x+r),  Zf = Zm + Zp - U, Yf(X) = Y- + Y+ - X(row);
//              H11 / H12 = Xf(Y+(Zf)) / Xf(Y-(Zf)),  Xf(X) = L(x) + L(x+r) - X(x);
//              H13 / H14 = Xf(Yf(Zm)) / Xf(Yf(Zp)).
// Window sums are re-formed from their register rings at every step (r <= 4), so no
// running sum drifts.  The yx-pass tile regions arrive by TMA (the tile grid is shifted by
// (4 - r % 4) % 4 columns so every box starts on 16 bytes).
#include <cstring>

#include "osbf.h"
#include "osbf_internal.h"

osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg);
void *osbf_ctx_workspace(osbf_ctx *ctx, int slot, size_t bytes, osbf_status *st);
void osbf_ctx_count_launches(osbf_ctx *ctx, int n);
void osbf_ctx_reset_launches(osbf_ctx *ctx);
unsigned int *osbf_ctx_err_word(osbf_ctx *ctx);

namespace osbf {
namespace v3 {

constexpr int TH = 32, TW = 64, SW = 32, NT = 64;

struct Vol {
    int D, H, W, FD, FH, FW, FWp;
    long long fplane;  // floats per padded volume (FD * FH * FWp)
};

// replicate padding of each D x H x W volume into its (D+2r) x (H+2r) x (W+2r) frame
__global__ void pad3d_kernel(const float *__restrict__ in, float *__restrict__ frame, Vol v, int R) {
    const int fy = blockIdx.y, fzp = blockIdx.z;
    const int fz = fzp % v.FD, p = fzp / v.FD;
    const int z = min(max(fz - R, 0), v.D - 1), y = min(max(fy - R, 0), v.H - 1);
    const float *src = in + (((long long)p * v.D + z) * v.H + y) * v.W;
    float *dst = frame + (long long)p * v.fplane + ((long long)fz * v.FH + fy) * v.FWp;
    for (int fx = blockIdx.x * blockDim.x + threadIdx.x; fx < v.FW; fx += gridDim.x * blockDim.x)
        dst[fx] = src[min(max(fx - R, 0), v.W - 1)];
}

// z-pass: thread = one (plane, y, x) column of the frame; ring over depths z-R..z+R.  The
// depths entering during a ring period (Q steps) are loaded a whole period ahead, so Q
// loads per thread are in flight while the current period is summed (one load per step,
// used at once, left the kernel waiting on memory latency).
template <int R>
__global__ void zpass_kernel(const float *__restrict__ U, float *__restrict__ Zm, float *__restrict__ Zp, Vol v) {
    constexpr int Q = 2 * R + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, p = blockIdx.z;
    if (x >= v.FW) return;
    const long long base = (long long)p * v.fplane + (long long)y * v.FWp + x;
    const long long zs = (long long)v.FH * v.FWp;  // floats per depth slice
    float ring[Q];  // ring[(z' mod Q)] = U(z') for z' in z-R..z+R (zero outside the volume)
#pragma unroll
    for (int k = 0; k < Q; ++k) ring[k] = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k)  // depths 0..R-1 enter ahead of the first output
        if (k < v.FD) ring[k % Q] = U[base + k * zs];
    // nxt[k]: the depth entering at step k of the next period (z0 + k + R), zero past the volume
    float nxt[Q];
    auto load_period = [&](int z0) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int zn = z0 + k + R;
            nxt[k] = zn < v.FD ? __ldg(U + base + (long long)zn * zs) : 0.f;
        }
    };
    load_period(0);
    for (int z0 = 0; z0 < v.FD; z0 += Q) {
        float cur[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) cur[k] = nxt[k];
        if (z0 + Q < v.FD) load_period(z0 + Q);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int z = z0 + k;
            if (z < v.FD) {
                ring[(k + R) % Q] = cur[k];  // depth z + R takes the slot depth z - R - 1 left
                float sm = ring[k], sp = ring[k];
#pragma unroll
                for (int j = 1; j <= R; ++j) {
                    sm += ring[(k + Q - j) % Q];
                    sp += ring[(k + j) % Q];
                }
                Zm[base + (long long)z * zs] = sm;
                Zp[base + (long long)z * zs] = sp;
            }
        }
    }
}

struct YXParams {
    float *dst;          // next frame, or the cropped output (dst_is_output)
    int dst_is_output;
    uint8_t *maps;       // this pass's maps (P x FD x FH x FW) or null
    Vol v;
    int tiles_x, tiles_y;
    int shift;           // tile k starts at frame column k * TW - shift: the boxes start on 16 bytes
    unsigned int *err;   // bit 0: a tile load did not land in time
};

// Width (floats) of the TMA boxes, also the row pitch of every shared field: the region
// TW + 2R plus pass H's float4 over-read, a multiple of 4 (16-byte rows) with
// pitch % 8 == 4, so the row-owner float4 loads of pass H are conflict-free.
__host__ __device__ constexpr int bx3(int R) {
    return ((TW + 2 * R + 4 + 3) / 4 * 4) % 8 == 4 ? (TW + 2 * R + 4 + 3) / 4 * 4 : (TW + 2 * R + 4 + 3) / 4 * 4 + 4;
}
__host__ __device__ constexpr int align128_3(int b) { return (b + 127) & ~127; }
// byte offsets: three boxes, three up-sum fields, the mbarrier
__host__ __device__ constexpr int box_bytes3(int R) { return (TH + 2 * R) * bx3(R) * 4; }
__host__ __device__ constexpr int off_a3(int R) { return 3 * align128_3(box_bytes3(R)); }
__host__ __device__ constexpr int smem3(int R) { return off_a3(R) + 3 * align128_3((TH + R) * bx3(R) * 4) + 16; }

// One CTA per (slice, 32 x 64 tile): the tile's region of U, Zm and Zp arrives by three
// TMA copies (zeros outside the frame), pass V forms the up-column sums, pass H selects.
template <int R, bool MAPS>
__global__ void __launch_bounds__(NT) yx_kernel(const __grid_constant__ CUtensorMap mU,
                                                const __grid_constant__ CUtensorMap mM,
                                                const __grid_constant__ CUtensorMap mP, const YXParams q) {
    constexpr int RH = TH + 2 * R, RW = TW + 2 * R, BX = bx3(R);
    constexpr int P = R + 1;
    constexpr float io = 1.0f / float((R + 1) * (R + 1) * (R + 1));
    constexpr float ih = 1.0f / float((R + 1) * (2 * R + 1) * (2 * R + 1));
    extern __shared__ __align__(128) unsigned char sm3[];
    float *bU = reinterpret_cast<float *>(sm3), *bM = reinterpret_cast<float *>(sm3 + align128_3(box_bytes3(R))),
          *bP = reinterpret_cast<float *>(sm3 + 2 * align128_3(box_bytes3(R)));
    constexpr int ab = align128_3((TH + R) * BX * 4);
    float *aU = reinterpret_cast<float *>(sm3 + off_a3(R)), *aM = reinterpret_cast<float *>(sm3 + off_a3(R) + ab),
          *aP = reinterpret_cast<float *>(sm3 + off_a3(R) + 2 * ab);
    const uint32_t bar = v2::smem_u32(sm3 + smem3(R) - 16);
    const Vol &v = q.v;
    const int tile = blockIdx.x, zp = blockIdx.y;
    const int z = zp % v.FD, p = zp / v.FD;
    const int ty0 = (tile / q.tiles_x) * TH, tx0 = (tile % q.tiles_x) * TW - q.shift;
    const long long slice = (long long)p * v.fplane + (long long)z * v.FH * v.FWp;

    if (threadIdx.x == 0) {
        v2::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        v2::fence_proxy_async();
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(3 * box_bytes3(R))
                     : "memory");
        const CUtensorMap *maps3[3] = {&mU, &mM, &mP};
        float *dst3[3] = {bU, bM, bP};
#pragma unroll
        for (int f = 0; f < 3; ++f)
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                "%3, %4}], [%5];" ::"r"(v2::smem_u32(dst3[f])),
                "l"(reinterpret_cast<uint64_t>(maps3[f])), "r"(tx0 - R), "r"(ty0 - R), "r"(zp), "r"(bar)
                : "memory");
    }
    __syncthreads();
    const bool timed_out = !v2::mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(timed_out)) {
        if (threadIdx.x == 0) {
            atomicOr(q.err, 1u);
            v2::mbar_wait_bounded(bar, 0);  // let late copies land before the CTA leaves
        }
        return;
    }

    // pass V: up-column sums (rows s-R..s) of the three fields, stored at row s - R; one
    // thread per column pair
    for (int c2 = threadIdx.x; 2 * c2 < RW; c2 += NT) {
        const int c = 2 * c2;
        float2 ru[P], rm[P], rp[P];
#pragma unroll
        for (int k = 0; k < P; ++k) ru[k] = rm[k] = rp[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < RH; ++s) {
            const int k = s % P;
            ru[k] = *reinterpret_cast<const float2 *>(bU + s * BX + c);
            rm[k] = *reinterpret_cast<const float2 *>(bM + s * BX + c);
            rp[k] = *reinterpret_cast<const float2 *>(bP + s * BX + c);
            if (s >= R) {
                float2 su = ru[0], smm = rm[0], spp = rp[0];
#pragma unroll
                for (int i = 1; i < P; ++i) {
                    su = __fadd2_rn(su, ru[i]);
                    smm = __fadd2_rn(smm, rm[i]);
                    spp = __fadd2_rn(spp, rp[i]);
                }
                *reinterpret_cast<float2 *>(aU + (s - R) * BX + c) = su;
                *reinterpret_cast<float2 *>(aM + (s - R) * BX + c) = smm;
                *reinterpret_cast<float2 *>(aP + (s - R) * BX + c) = spp;
            }
        }
    }
    __syncthreads();

    // pass H: lane = output row, warp = 32-column segment; shared loads as float4 groups
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = lane, xs = warp * SW;
    constexpr int NS = SW + 2 * R;
    const float4 *gau = reinterpret_cast<const float4 *>(aU + y * BX + xs);
    const float4 *gbu = reinterpret_cast<const float4 *>(aU + (y + R) * BX + xs);
    const float4 *gam = reinterpret_cast<const float4 *>(aM + y * BX + xs);
    const float4 *gbm = reinterpret_cast<const float4 *>(aM + (y + R) * BX + xs);
    const float4 *gap = reinterpret_cast<const float4 *>(aP + y * BX + xs);
    const float4 *gbp = reinterpret_cast<const float4 *>(aP + (y + R) * BX + xs);
    const float4 *gcu = reinterpret_cast<const float4 *>(bU + (y + R) * BX + xs);
    const float4 *gcm = reinterpret_cast<const float4 *>(bM + (y + R) * BX + xs);
    const float4 *gcp = reinterpret_cast<const float4 *>(bP + (y + R) * BX + xs);
    float4 vau, vbu, vam, vbm, vap, vbp, vcu, vcm, vcp;
    // nine row fields, by step t (region column xs + t): 0 Y-(Zm) 1 Y+(Zm) 2 Y-(Zp) 3 Y+(Zp)
    // 4 Yf(Zf) 5 Y+(Zf) 6 Y-(Zf) 7 Yf(Zm) 8 Yf(Zp)
    float rf[9][P];  // field values of the last P columns
    float lh[9][P];  // their left sums L at the last P columns
#pragma unroll
    for (int f = 0; f < 9; ++f)
#pragma unroll
        for (int k = 0; k < P; ++k) rf[f][k] = lh[f][k] = 0.f;
    float ucol[P];
    const int fy = ty0 + y;
    // the sweep runs in blocks of UN steps, a multiple of the ring period and of the 4-step
    // load group, so ring slots and vector lanes stay static while the code stays within
    // the instruction cache (a fully unrolled sweep stalled on instruction fetch)
    constexpr int UN = (P % 4 == 0) ? P : (P % 2 == 0 ? 2 * P : 4 * P);
#pragma unroll 1
    for (int t0 = 0; t0 < NS; t0 += UN) {
#pragma unroll
    for (int i = 0; i < UN; ++i) {
        const int t = t0 + i;
        if (t >= NS) break;
        const int k = i % P, j = i & 3;
        if (j == 0) {
            const int g = t >> 2;
            vau = gau[g];
            vbu = gbu[g];
            vam = gam[g];
            vbm = gbm[g];
            vap = gap[g];
            vbp = gbp[g];
            vcu = gcu[g];
            vcm = gcm[g];
            vcp = gcp[g];
        }
        const float amu = f4get(vau, j), bpu = f4get(vbu, j), amm = f4get(vam, j), bpm = f4get(vbm, j);
        const float amp = f4get(vap, j), bpp = f4get(vbp, j);
        const float uc = f4get(vcu, j), mc = f4get(vcm, j), pc = f4get(vcp, j);
        const float zf = mc + pc - uc;
        const float ymzf = amm + amp - amu, ypzf = bpm + bpp - bpu;
        float fv[9];
        fv[0] = amm;
        fv[1] = bpm;
        fv[2] = amp;
        fv[3] = bpp;
        fv[4] = ymzf + ypzf - zf;
        fv[5] = ypzf;
        fv[6] = ymzf;
        fv[7] = amm + bpm - mc;
        fv[8] = amp + bpp - pc;
        ucol[k] = uc;
#pragma unroll
        for (int f = 0; f < 9; ++f) {
            rf[f][k] = fv[f];
            float sum = fv[f];
#pragma unroll
            for (int i = 1; i < P; ++i) sum += rf[f][(k + P - i) % P];
            lh[f][k] = sum;  // L at column t (valid once t >= R)
        }
        if (t >= 2 * R) {
            const int sl = (k + P - R) % P;  // column x = t - R: the output pixel's column
            const float u = ucol[sl];
            float mean[15];
            mean[1] = lh[1][sl] * io;  // O1: z-, y+, x-
            mean[2] = lh[1][k] * io;   // O2: z-, y+, x+
            mean[3] = lh[0][k] * io;   // O3: z-, y-, x+
            mean[4] = lh[0][sl] * io;  // O4: z-, y-, x-
            mean[5] = lh[3][sl] * io;  // O5..O8: z+ with N1..N4
            mean[6] = lh[3][k] * io;
            mean[7] = lh[2][k] * io;
            mean[8] = lh[2][sl] * io;
            mean[9] = lh[4][sl] * ih;                            // H9: x-
            mean[10] = lh[4][k] * ih;                            // H10: x+
            mean[11] = (lh[5][sl] + lh[5][k] - rf[5][sl]) * ih;  // H11: y+
            mean[12] = (lh[6][sl] + lh[6][k] - rf[6][sl]) * ih;  // H12: y-
            mean[13] = (lh[7][sl] + lh[7][k] - rf[7][sl]) * ih;  // H13: z-
            mean[14] = (lh[8][sl] + lh[8][k] - rf[8][sl]) * ih;  // H14: z+
            // first argmin |mean_w - u| as a tournament: in every pick the left operand
            // holds the earlier windows and keeps ties, so the first index still wins
            float d[15];
            int id[15];
#pragma unroll
            for (int w = 1; w <= 14; ++w) {
                d[w] = mean[w] - u;
                id[w] = w;
            }
            auto pick = [&](int a, int b) {  // into slot a
                const bool take = fabsf(d[b]) < fabsf(d[a]);
                d[a] = take ? d[b] : d[a];
                if (MAPS) id[a] = take ? id[b] : id[a];
            };
            pick(1, 2); pick(3, 4); pick(5, 6); pick(7, 8); pick(9, 10); pick(11, 12); pick(13, 14);
            pick(1, 3); pick(5, 7); pick(9, 11);
            pick(1, 5); pick(9, 13);
            pick(1, 9);
            const float best = d[1];
            const int m = id[1];
            const int fx = tx0 + xs + t - 2 * R;
            if (fy < v.FH && (unsigned)fx < (unsigned)v.FW) {
                const float outv = u + best;
                if (q.dst_is_output) {
                    const int oz = z - R, oy = fy - R, ox = fx - R;
                    if ((unsigned)oz < (unsigned)v.D && (unsigned)oy < (unsigned)v.H && (unsigned)ox < (unsigned)v.W)
                        q.dst[(((long long)p * v.D + oz) * v.H + oy) * v.W + ox] = outv;
                } else {
                    q.dst[slice + (long long)fy * v.FWp + fx] = outv;
                }
                if (MAPS) q.maps[(((long long)p * v.FD + z) * v.FH + fy) * v.FW + fx] = (uint8_t)m;
            }
        }
    }
    }
}

template <int R>
cudaError_t launch_yx(const CUtensorMap &mU, const CUtensorMap &mM, const CUtensorMap &mP, const YXParams &q,
                      int nslices, cudaStream_t s) {
    const int bytes = smem3(R);
    auto kern = q.maps ? yx_kernel<R, true> : yx_kernel<R, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    kern<<<dim3(q.tiles_x * q.tiles_y, nslices), NT, bytes, s>>>(mU, mM, mP, q);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_z(const float *U, float *Zm, float *Zp, const Vol &v, int P, cudaStream_t s) {
    zpass_kernel<R><<<dim3((v.FW + 127) / 128, v.FH, P), 128, 0, s>>>(U, Zm, Zp, v);
    return cudaGetLastError();
}

}  // namespace v3
}  // namespace osbf

using namespace osbf;

extern "C" osbf_status osbf_filter_3d(osbf_ctx *ctx, const float *in, float *out, int N, int C, int D, int H, int W,
                                     int r, int iters, uint8_t *maps, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    osbf_ctx_reset_launches(ctx);
    if (!in || !out) return osbf_ctx_fail(ctx, OSBF_EINVAL, "null pointer");
    if (N <= 0 || C <= 0 || D <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0)
        return osbf_ctx_fail(ctx, OSBF_EINVAL, "N, C, D, H, W must be positive; r, iters >= 0");
    if (r > OSBF_MAX_RADIUS_3D) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "r exceeds OSBF_MAX_RADIUS_3D");
    const long long P = (long long)N * C;
    const size_t bytes = sizeof(float) * (size_t)P * D * H * W;
    if ((const char *)in < (const char *)out + bytes && (const char *)out < (const char *)in + bytes)
        return osbf_ctx_fail(ctx, OSBF_EINVAL, "in and out overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0 || iters == 0) {
        if (cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "copy failed");
        if (maps && iters > 0) {  // every window is the voxel: O1, first in the order
            const long long n = (long long)iters * P * (D + 2 * r) * (H + 2 * r) * (W + 2 * r);
            if (launch_fill_u8(maps, 1, n, s) != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, "fill failed");
        }
        osbf_ctx_count_launches(ctx, 1);
        return OSBF_OK;
    }
    v3::Vol v;
    v.D = D;
    v.H = H;
    v.W = W;
    v.FD = D + 2 * r;
    v.FH = H + 2 * r;
    v.FW = W + 2 * r;
    v.FWp = (v.FW + 31) / 32 * 32;
    v.fplane = (long long)v.FD * v.FH * v.FWp;
    if ((long long)v.FH > 65535 || P * v.FD > 65535)
        return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "volume too large for the 3D launch grid");
    const size_t fbytes = sizeof(float) * (size_t)P * v.fplane;
    osbf_status st;
    float *fr[2], *Zm, *Zp;
    for (int k = 0; k < 2; ++k) {
        fr[k] = (float *)osbf_ctx_workspace(ctx, k, fbytes, &st);
        if (st) return st;
    }
    Zm = (float *)osbf_ctx_workspace(ctx, 2, fbytes, &st);
    if (st) return st;
    Zp = (float *)osbf_ctx_workspace(ctx, 3, fbytes, &st);
    if (st) return st;
    v3::pad3d_kernel<<<dim3((v.FW + 255) / 256 < 8 ? (v.FW + 255) / 256 : 8, v.FH, (unsigned)(P * v.FD)), 256, 0,
                       s>>>(in, fr[0], v, r);
    if (cudaGetLastError() != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, "3D pad launch failed");
    osbf_ctx_count_launches(ctx, 1);
    int cur = 0;
    const long long mstride = P * v.FD * v.FH * v.FW;
    for (int pass = 0; pass < iters; ++pass) {
        cudaError_t e = cudaErrorInvalidValue;
        switch (r) {
        case 1: e = v3::launch_z<1>(fr[cur], Zm, Zp, v, (int)P, s); break;
        case 2: e = v3::launch_z<2>(fr[cur], Zm, Zp, v, (int)P, s); break;
        case 3: e = v3::launch_z<3>(fr[cur], Zm, Zp, v, (int)P, s); break;
        case 4: e = v3::launch_z<4>(fr[cur], Zm, Zp, v, (int)P, s); break;
        }
        if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
        v3::YXParams q;
        std::memset(&q, 0, sizeof q);
        const bool last = pass == iters - 1;
        q.dst = last ? out : fr[1 - cur];
        q.dst_is_output = last ? 1 : 0;
        q.maps = maps ? maps + pass * mstride : nullptr;
        q.v = v;
        q.shift = (4 - r % 4) % 4;
        q.tiles_x = (v.FW - 1 + q.shift) / v3::TW + 1;
        q.tiles_y = (v.FH + v3::TH - 1) / v3::TH;
        q.err = osbf_ctx_err_word(ctx);
        const int nslices = (int)(P * v.FD);
        // the three fields as P*FD slices of FH x FW (row pitch FWp); boxes of the tile region
        const int bx = r == 1 ? v3::bx3(1) : r == 2 ? v3::bx3(2) : r == 3 ? v3::bx3(3) : v3::bx3(4);
        CUtensorMap mU, mM, mP;
        if (!encode_frame_map(&mU, Storage::F32, fr[cur], v.FW, v.FH, nslices, v.FWp, bx, v3::TH + 2 * r) ||
            !encode_frame_map(&mM, Storage::F32, Zm, v.FW, v.FH, nslices, v.FWp, bx, v3::TH + 2 * r) ||
            !encode_frame_map(&mP, Storage::F32, Zp, v.FW, v.FH, nslices, v.FWp, bx, v3::TH + 2 * r))
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "cuTensorMapEncodeTiled failed (3D fields)");
        switch (r) {
        case 1: e = v3::launch_yx<1>(mU, mM, mP, q, nslices, s); break;
        case 2: e = v3::launch_yx<2>(mU, mM, mP, q, nslices, s); break;
        case 3: e = v3::launch_yx<3>(mU, mM, mP, q, nslices, s); break;
        case 4: e = v3::launch_yx<4>(mU, mM, mP, q, nslices, s); break;
        }
        if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
        osbf_ctx_count_launches(ctx, 2);
        cur = 1 - cur;
    }
    return OSBF_OK;
}
