// osbf_fwd.cuh -- forward tile kernel of the One-Sided Box Filter for sm_103a.
//
// One CTA owns a TH x TW tile of one padded frame and runs D fused passes of
// Algorithm 2 on it in shared memory (temporal blocking): it loads the tile with
// a halo of D*r rows and >= D*r columns, and every pass shrinks the valid region
// by r on each side.  Every pass is two sweeps over shared memory:
//
//   pass V  (one thread per column, sweeping down):  a(y, x) = sum_{y-r..y} U(., x)
//           -- the "up" column sums; a(y + r, x) is the "down" sum b(y, x).
//   pass H  (one thread per row segment, sweeping right): the left row sums of
//           a, b and U, AL(x) = sum_{x-r..x} a, BL, UL, kept in register rings, give
//           all eight window sums of Eq. (6)-(13) at (y, x) from values at x and x+r:
//             N4 = AL(x)     N3 = AL(x+r)   N1 = BL(x)     N2 = BL(x+r)
//             N5 = AL(x) + BL(x) - UL(x)       N6 = AL(x+r) + BL(x+r) - UL(x+r)
//             N8 = AL(x) + AL(x+r) - a(x)      N7 = BL(x) + BL(x+r) - b(x)
//           then d_i = S_i / n_i - U, m = first argmin |d_i| in the tie order, and
//           U' = U + d_m (Algorithm 2), zero outside the padded frame (the appendix's
//           'same' convolution on the padded image).
//
// Both sweeps are running sums (O(1) per pixel in r, as the paper's complexity
// section requires): a value enters a ring and leaves it r+1 steps later.  The
// rings are register arrays indexed by compile-time slots, so the radius is a
// template parameter.  Both sums are re-formed from their ring once per ring period
// (every step for r <= 3), so FP32 drift stays bounded by a few roundings: the
// selection must see |d_i| to well within the 1e-6 tie band.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace osbf {

// ----------------------------------------------------------------------------------
// tile geometry (shared by host and device)
// ----------------------------------------------------------------------------------
constexpr int kTH = 32;   // tile rows
constexpr int kTW = 128;  // tile columns
constexpr int kSW = 32;   // columns per pass-H segment
constexpr int kNT = 128;  // threads per CTA

struct Layout {
    int EY, EX;    // halo rows / columns of the loaded region
    int RH0, RW0;  // loaded region
    int pitch;     // floats per shared-memory row (pitch/4 odd: conflict-free 16-byte row-owner access)
    int offU0, offU1, offA;
    int floats;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// xalign: horizontal halo rounded up to this many elements (16-byte global access).
__host__ __device__ inline Layout make_layout(int R, int D, int xalign) {
    Layout L;
    L.EY = D * R;
    L.EX = round_up(D * R, xalign);
    L.RH0 = kTH + 2 * L.EY;
    L.RW0 = kTW + 2 * L.EX;
    int pitch = L.RW0 + 8;  // row sweeps read (and write) up to 6 columns past the region
    if (pitch % 8 == 0) pitch += 4;
    L.pitch = pitch;
    L.offU0 = 0;
    L.offA = L.RH0 * pitch;
    L.offU1 = L.offA + (L.RH0 - R) * pitch;
    L.floats = L.offU1 + (L.RH0 - 2 * R) * pitch + 16;  // tail: the last row's sweep over-read
    return L;
}

struct FwdParams {
    const void *src;        // group input: the caller's image (src_is_input) or a padded frame
    void *dst;              // group output: a padded frame or the caller's output (dst_is_output)
    uint8_t *maps;          // selection maps [iters][P][FH][map_pitch] or null
    int map_pitch;          // bytes per map row
    long long src_plane, dst_plane;  // elements per plane
    int src_pitch, dst_pitch;        // elements per row
    int H, W, FH, FW;
    int src_is_input, dst_is_output;
    int D;                  // passes fused in this launch
    int map_iter0;          // global pass index of this launch's first pass
    long long map_iter_stride, map_plane;
    int ty_off, tx_off;     // tile index offsets (final launches skip tiles without output pixels)
};

// ----------------------------------------------------------------------------------
// storage types
// ----------------------------------------------------------------------------------
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(uint8_t v) { return (float)v; }

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// value as it will be stored (rounded to the storage type after every pass)
template <typename T> __device__ __forceinline__ float storage_round(float v) { return to_f(from_f<T>(v)); }
template <> __device__ __forceinline__ float storage_round<float>(float v) { return v; }

__device__ __forceinline__ float f4get(const float4 &v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// window index at tie-order position k (paper: N1..N8; appendix: N6 N5 N7 N8 N2 N1 N3 N4)
template <bool TIE_APP> __host__ __device__ constexpr int tie_window(int k) {
    return TIE_APP ? (k == 0 ? 6 : k == 1 ? 5 : k == 2 ? 7 : k == 3 ? 8 : k == 4 ? 2 : k == 5 ? 1 : k == 6 ? 3 : 4)
                   : k + 1;
}

// keep (da, ia) unless b is strictly closer: left operand (lower tie position) wins ties
template <bool IDX> __device__ __forceinline__ void pick(float &da, int &ia, float db, int ib) {
    const bool take = fabsf(db) < fabsf(da);
    da = take ? db : da;
    if (IDX) ia = take ? ib : ia;
}

// FP32 selection of Algorithm 2.  S[1..8] window sums, u the centre value.
template <int R, bool TIE_APP, bool IDX>
__device__ __forceinline__ void select_f32(const float (&S)[9], float u, float &out, int &m) {
    constexpr float inv_q = 1.0f / float((R + 1) * (R + 1));
    constexpr float inv_h = 1.0f / float((R + 1) * (2 * R + 1));
    float d[8];
    int id[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = tie_window<TIE_APP>(k);
        d[k] = fmaf(S[i], i <= 4 ? inv_q : inv_h, -u);
        id[k] = i;
    }
    pick<IDX>(d[0], id[0], d[1], id[1]);
    pick<IDX>(d[2], id[2], d[3], id[3]);
    pick<IDX>(d[4], id[4], d[5], id[5]);
    pick<IDX>(d[6], id[6], d[7], id[7]);
    pick<IDX>(d[0], id[0], d[2], id[2]);
    pick<IDX>(d[4], id[4], d[6], id[6]);
    pick<IDX>(d[0], id[0], d[4], id[4]);
    out = u + d[0];
    m = id[0];
}

// Exact 8-bit selection: integer sums, |S_i - n_i U| / n_i compared by
// cross-multiplication in int64; output the correctly rounded S_m / n_m.
template <int R, bool TIE_APP>
__device__ __forceinline__ void select_u8(const float (&S)[9], float u, float &out, int &m) {
    constexpr long long nq = (long long)(R + 1) * (R + 1);
    constexpr long long nh = (long long)(R + 1) * (2 * R + 1);
    const long long ui = (long long)__float2int_rn(u);
    long long sc[8];
    int id[8];
    long long sm[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = tie_window<TIE_APP>(k);
        const long long s = (long long)__float2int_rn(S[i]);
        const long long n = i <= 4 ? nq : nh;
        long long dev = s - n * ui;
        dev = dev < 0 ? -dev : dev;
        sc[k] = dev * (i <= 4 ? nh : nq);  // |d_i| * nq * nh
        id[k] = i;
        sm[k] = s;
    }
    long long sc_best = sc[0], s_best = sm[0];
    int i_best = id[0];
#pragma unroll
    for (int k = 1; k < 8; ++k)
        if (sc[k] < sc_best) {  // strictly smaller: the first position in tie order wins
            sc_best = sc[k];
            s_best = sm[k];
            i_best = id[k];
        }
    out = __fdiv_rn((float)s_best, (float)(i_best <= 4 ? nq : nh));
    m = i_best;
}

// ----------------------------------------------------------------------------------
// load the region of U^0 into shared memory (zero outside the padded frame)
// ----------------------------------------------------------------------------------
template <int R, typename TIn>
__device__ __forceinline__ void load_region(const FwdParams &p, const Layout &L, float *__restrict__ U0, int plane,
                                            int ty0, int tx0) {
    const TIn *src = reinterpret_cast<const TIn *>(p.src) + (long long)plane * p.src_plane;
    const int fy0 = ty0 - L.EY, fx0 = tx0 - L.EX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < L.RH0; y += kNT / 32) {
        const int fy = fy0 + y;
        const bool yin = (unsigned)fy < (unsigned)p.FH;
        int sy = fy;
        if (p.src_is_input) sy = min(max(fy - R, 0), p.H - 1);  // replicate padding
        const TIn *srow = src + (long long)(yin ? sy : 0) * p.src_pitch;
        float *drow = U0 + y * L.pitch;
        for (int x = lane; x < L.RW0; x += 32) {
            const int fx = fx0 + x;
            float v = 0.f;
            if (yin && (unsigned)fx < (unsigned)p.FW) {
                const int sx = p.src_is_input ? min(max(fx - R, 0), p.W - 1) : fx;
                v = to_f(srow[sx]);
            }
            drow[x] = v;
        }
    }
}

// ----------------------------------------------------------------------------------
// pass V: a(y) = sum_{y-R..y} U(., x) for region rows y in [R, RH), stored at A[(y-R)]
// ----------------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void pass_v(const float *__restrict__ U, float *__restrict__ A, int RH, int RW, int pitch) {
    constexpr int P = R + 1;
    const int na = RH - R;
    int nch = (2 * kNT) / RW;
    const int maxch = na / (2 * R > 8 ? 2 * R : 8);
    if (nch > maxch) nch = maxch;
    if (nch < 1) nch = 1;
    const int ch = (na + nch - 1) / nch;
    for (int item = threadIdx.x; item < RW * nch; item += kNT) {
        const int c = item % RW, kc = item / RW;
        const int ya0 = kc * ch;
        const int ya1 = min(na, ya0 + ch);
        if (ya0 >= ya1) continue;
        const int n = ya1 - ya0 + R;
        const float *col = U + ya0 * pitch + c;
        float *acol = A + ya0 * pitch + c;
        float ring[P];
#pragma unroll
        for (int k = 0; k < P; ++k) ring[k] = 0.f;
        float acc = 0.f;
        for (int s0 = 0; s0 < n; s0 += P) {
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int s = s0 + k;
                if (s < n) {
                    const float v = col[s * pitch];
                    acc += v - ring[k];
                    ring[k] = v;
                    if (k == P - 1) {  // the ring holds exactly the window: re-form the sum
                        float t = ring[0];
#pragma unroll
                        for (int i = 1; i < P; ++i) t += ring[i];
                        acc = t;
                    }
                    if (s >= R) acol[(s - R) * pitch] = acc;
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------------
// pass H: one warp = 32 consecutive rows of one SW-column segment; one lane = one row
// ----------------------------------------------------------------------------------
struct PassHGeom {
    int RHo, RWo;       // U^j region
    int fy0, fx0;       // frame coordinates of the U^j region origin
    int FH, FW;
    int iy0, iy1, ix0, ix1;  // tile interior in U^j region coordinates (map writes)
    int MP;                  // map row pitch (bytes)
};

template <int R, typename TSt, bool TIE_APP, bool MAPS, bool U8X>
__device__ __forceinline__ void pass_h(const float *__restrict__ Uin, const float *__restrict__ A,
                                       float *__restrict__ Uout, int pitch, const PassHGeom g,
                                       uint8_t *__restrict__ mplane) {
    constexpr int P = (R + 1 + 3) & ~3;  // ring period: >= R+1 and a multiple of 4
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrb = (g.RHo + 31) >> 5;
    const int nseg = (g.RWo + kSW - 1) / kSW;
    for (int item = warp; item < nrb * nseg; item += kNT / 32) {
        const int rbk = item % nrb, seg = item / nrb;
        const int yo = rbk * 32 + lane;
        const bool row_ok = yo < g.RHo;
        const int yr = row_ok ? yo : g.RHo - 1;
        const int xs = seg * kSW;
        const float *arow = A + yr * pitch + xs;
        const float *brow = A + (yr + R) * pitch + xs;
        const float *urow = Uin + (yr + R) * pitch + xs;
        float *orow = Uout + yr * pitch + xs;
        const int nout = min(kSW, g.RWo - xs);
        const int nst = ((nout + 3) & ~3) + 2 * R;
        const int fy = g.fy0 + yo;
        const bool row_in = row_ok && (unsigned)fy < (unsigned)g.FH;
        const bool row_map = MAPS && row_in && yo >= g.iy0 && yo < g.iy1 && mplane != nullptr;
        float ra[P], rb[P], ru[P], hA[P], hB[P], hU[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            ra[k] = 0.f; rb[k] = 0.f; ru[k] = 0.f;
            hA[k] = 0.f; hB[k] = 0.f; hU[k] = 0.f;
        }
        float AL = 0.f, BL = 0.f, UL = 0.f;
        float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va, vu = va;
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        for (int t0 = 0; t0 < nst; t0 += P) {
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int t = t0 + k;
                if (t < nst) {
                    if ((k & 3) == 0) {
                        va = *reinterpret_cast<const float4 *>(arow + t);
                        vb = *reinterpret_cast<const float4 *>(brow + t);
                        vu = *reinterpret_cast<const float4 *>(urow + t);
                    }
                    const float a = f4get(va, k & 3), b = f4get(vb, k & 3), u = f4get(vu, k & 3);
                    const int so = (k + 2 * P - R - 1) % P;  // value leaving the window (t - R - 1)
                    if (R <= 3 || k == P - 1) {
                        // direct sum of the ring's last R+1 entries: for small r it costs no more
                        // than the running update, for large r it resets the FP32 drift once
                        // per ring period
                        ra[k] = a; rb[k] = b; ru[k] = u;
                        AL = ra[k]; BL = rb[k]; UL = ru[k];
#pragma unroll
                        for (int i = 1; i <= R; ++i) {
                            const int si = (k + P - i) % P;
                            AL += ra[si];
                            BL += rb[si];
                            UL += ru[si];
                        }
                    } else {
                        AL += a - ra[so];
                        BL += b - rb[so];
                        UL += u - ru[so];
                        ra[k] = a; rb[k] = b; ru[k] = u;
                    }
                    hA[k] = AL; hB[k] = BL; hU[k] = UL;
                    if (t >= 2 * R) {
                        const int sl = (k + P - R) % P;  // column x = t - R
                        const float ALx = hA[sl], BLx = hB[sl], ULx = hU[sl];
                        float S[9];
                        S[0] = 0.f;
                        S[1] = BLx;                 // N1: down-left quadrant
                        S[2] = BL;                  // N2: down-right quadrant
                        S[3] = AL;                  // N3: up-right quadrant
                        S[4] = ALx;                 // N4: up-left quadrant
                        S[5] = ALx + BLx - ULx;     // N5: left half
                        S[6] = AL + BL - UL;        // N6: right half
                        S[7] = BLx + BL - rb[sl];   // N7: down half
                        S[8] = ALx + AL - ra[sl];   // N8: up half
                        const float ux = ru[sl];
                        float outv;
                        int m;
                        if (U8X)
                            select_u8<R, TIE_APP>(S, ux, outv, m);
                        else
                            select_f32<R, TIE_APP, MAPS>(S, ux, outv, m);
                        const int xo = xs + t - 2 * R;
                        const int fx = g.fx0 + xo;
                        const bool in = row_in && (unsigned)fx < (unsigned)g.FW;
                        outv = in ? storage_round<TSt>(outv) : 0.f;
                        const int oi = (k - 2 * R) & 3;
                        o[oi] = outv;
                        if (MAPS) {
                            if (row_map && in && xo >= g.ix0 && xo < g.ix1) mplane[(long long)fy * g.MP + fx] = (uint8_t)m;
                        }
                        if (oi == 3 && row_ok)
                            *reinterpret_cast<float4 *>(orow + (t - 2 * R - 3)) = make_float4(o[0], o[1], o[2], o[3]);
                    }
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------------
// the kernel
// ----------------------------------------------------------------------------------
template <typename TIn> struct XAlign { static constexpr int v = 16 / sizeof(TIn) < 4 ? 4 : 16 / sizeof(TIn); };

template <typename TIn, typename TSt, int R, bool TIE_APP, bool MAPS, bool U8X>
__global__ void __launch_bounds__(kNT, 3) osbf_fwd_tile(const FwdParams p) {
    extern __shared__ __align__(16) float smem[];
    const Layout L = make_layout(R, p.D, XAlign<TSt>::v);
    const int plane = blockIdx.z;
    const int ty0 = (blockIdx.y + p.ty_off) * kTH, tx0 = (blockIdx.x + p.tx_off) * kTW;
    float *U0 = smem + L.offU0;
    float *U1 = smem + L.offU1;
    float *A = smem + L.offA;

    load_region<R, TIn>(p, L, U0, plane, ty0, tx0);
    __syncthreads();

    for (int j = 1; j <= p.D; ++j) {
        const float *Uin = (j & 1) ? U0 : U1;
        float *Uout = (j & 1) ? U1 : U0;
        const int RH = L.RH0 - 2 * (j - 1) * R, RW = L.RW0 - 2 * (j - 1) * R;
        pass_v<R>(Uin, A, RH, RW, L.pitch);
        __syncthreads();
        PassHGeom g;
        g.RHo = RH - 2 * R;
        g.RWo = RW - 2 * R;
        g.fy0 = ty0 - (L.EY - j * R);
        g.fx0 = tx0 - (L.EX - j * R);
        g.FH = p.FH;
        g.FW = p.FW;
        g.iy0 = L.EY - j * R;
        g.iy1 = g.iy0 + kTH;
        g.ix0 = L.EX - j * R;
        g.ix1 = g.ix0 + kTW;
        g.MP = p.map_pitch;
        uint8_t *mplane = nullptr;
        if (MAPS && p.maps)
            mplane = p.maps + (long long)(p.map_iter0 + j - 1) * p.map_iter_stride + (long long)plane * p.map_plane;
        pass_h<R, TSt, TIE_APP, MAPS, U8X>(Uin, A, Uout, L.pitch, g, mplane);
        __syncthreads();
    }

    // store the tile interior of U^D
    const float *UD = (p.D & 1) ? U1 : U0;
    const int cx = L.EX - p.D * R;
    TSt *dst = reinterpret_cast<TSt *>(p.dst) + (long long)plane * p.dst_plane;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < kTH; y += kNT / 32) {
        const int fy = ty0 + y;
        if (fy >= p.FH) break;
        const float *srow = UD + y * L.pitch + cx;
        if (p.dst_is_output) {
            const int oy = fy - R;
            if (oy < 0 || oy >= p.H) continue;
            TSt *drow = dst + (long long)oy * p.dst_pitch;
            for (int x = lane; x < kTW; x += 32) {
                const int ox = tx0 + x - R;
                if (ox >= 0 && ox < p.W) drow[ox] = from_f<TSt>(srow[x]);
            }
        } else {
            TSt *drow = dst + (long long)fy * p.dst_pitch;
            for (int x = lane; x < kTW; x += 32) {
                const int fx = tx0 + x;
                if (fx < p.FW) drow[fx] = from_f<TSt>(srow[x]);
            }
        }
    }
}

template <typename TIn, typename TSt>
inline size_t fwd_smem_bytes(int R, int D) {
    return sizeof(float) * (size_t)make_layout(R, D, XAlign<TSt>::v).floats;
}

template <typename TIn, typename TSt, int R, bool TIE_APP, bool MAPS, bool U8X>
cudaError_t launch_fwd_tile(const FwdParams &p, dim3 grid, cudaStream_t stream) {
    const size_t smem = fwd_smem_bytes<TIn, TSt>(R, p.D);
    auto kern = osbf_fwd_tile<TIn, TSt, R, TIE_APP, MAPS, U8X>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kNT, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace osbf
