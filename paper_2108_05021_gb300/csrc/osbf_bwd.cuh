// osbf_bwd.cuh -- adjoint (backward) tile kernel of the One-Sided Box Filter (sm_103a).
//
// With every pixel's selection m(p) frozen, one pass of Algorithm 2 is linear:
//   U'(p) = (1/n_m(p)) * sum_{o in O_m(p)} U(p + o)       (zero outside the padded frame),
// where O_k are the offsets of window N_k (Eq. (6)-(13)).  Its transpose is
//   g_in(q) = sum_k sum_{o in O_k} G_k(q - o),   G_k(p) = [m(p) = k] g(p) / n_k,
// i.e. every window type contributes a box sum of its masked field over the point-
// mirrored window.  Written with the up column sum Vup(F)(y) = sum_{y-r..y} F and the
// left row sum HL(F)(x) = sum_{x-r..x} F, the eight mirrored windows regroup into
//   g_in(y, x) = HL[F1](x) + HL[F2](x + r) - F3(x)
//   F1(y) = Vup(c1)(y) + Vup(c2)(y + r) - G_6(y)      c1 = G_2 + G_6 + G_7,  c2 = G_3 + G_6 + G_8
//   F2(y) = Vup(c3)(y) + Vup(c4)(y + r) - G_5(y)      c3 = G_1 + G_5 + G_7,  c4 = G_4 + G_5 + G_8
//   F3(y) = Vup(c5)(y) + Vup(c6)(y + r)               c5 = G_7,              c6 = G_8
// (mirrored N2 / N3 / N6 / N7 / N8 evaluate HL at x, mirrored N1 / N4 / N5 / N7 / N8 at
// x + r; the full-width rows of N7 / N8 subtract their centre column once).
// One CTA owns a 32 x 128 tile: pass V sweeps columns computing the six column sums,
// pass H sweeps row segments computing the two left sums -- the same O(1)-in-r
// structure as the forward.  One launch per pass (the forward's maps of that pass).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace osbf {
namespace bwd {

constexpr int TH = 32, TW = 128, SW = 32, NT = 128;

struct BwdParams {
    const float *gsrc;       // incoming gradient: a padded frame, or the caller's grad_out (src_is_output)
    int src_is_output;       // 1: gsrc is H x W (embed into a zero frame); 0: frame with pitch src_pitch
    long long src_plane;
    int src_pitch;
    const uint8_t *maps;     // this pass's selections, P x FH x FW
    float *gdst;             // outgoing gradient frame (pitch dst_pitch)
    long long dst_plane;
    int dst_pitch;
    int H, W, FH, FW, R;
};

struct BLayout {
    int RH, RW, PG, PF;  // region rows / cols; float pitch of the g box; float2 pitch of the (F1, F2) field
    int off_g, off_m, off_f12, off_f3, bytes;
};

__host__ __device__ inline BLayout make_blayout(int R) {
    BLayout L;
    L.RH = TH + 2 * R;
    L.RW = TW + 2 * R;
    L.PG = L.RW + 9;  // odd: lanes = rows read F3 conflict-free
    if ((L.PG & 1) == 0) ++L.PG;
    L.PF = L.PG;      // odd float2 pitch: conflict-free 8-byte row-owner loads
    L.off_g = 0;
    L.off_m = L.off_g + L.RH * L.PG * 4;
    L.off_f12 = (L.off_m + L.RH * L.PG + 15) & ~15;
    L.off_f3 = L.off_f12 + TH * L.PF * 8;
    L.bytes = L.off_f3 + TH * L.PG * 4 + 64;
    return L;
}

// which column-sum inputs c1..c6 receive G_m (bit j-1 for c_j), and whether it is G_5 / G_6
__device__ __forceinline__ unsigned cmask(int m) {
    // m:      1        2        3        4        5         6         7          8
    // c-bits: c3       c1       c2       c4       c3,c4     c1,c2     c1,c3,c5   c2,c4,c6
    const unsigned long long lut = (0x04ull << 8) | (0x01ull << 16) | (0x02ull << 24) | (0x08ull << 32) |
                                   (0x0Cull << 40) | (0x03ull << 48) | (0x15ull << 56);
    return m == 8 ? 0x2Au : (unsigned)(lut >> (8 * m)) & 0xFFu;
}

template <int R>
__global__ void __launch_bounds__(NT, 2) osbf_bwd_tile(const BwdParams p) {
    extern __shared__ __align__(16) unsigned char bsm[];
    const BLayout L = make_blayout(R);
    float *gb = reinterpret_cast<float *>(bsm + L.off_g);
    uint8_t *mb = bsm + L.off_m;
    float2 *F12 = reinterpret_cast<float2 *>(bsm + L.off_f12);
    float *F3 = reinterpret_cast<float *>(bsm + L.off_f3);
    constexpr float iq = 1.0f / float((R + 1) * (R + 1));
    constexpr float ih = 1.0f / float((R + 1) * (2 * R + 1));

    const int plane = blockIdx.z;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int fy0 = ty0 - R, fx0 = tx0 - R;  // frame coordinates of the region origin
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // ---- load g and the selections of the region (zero outside the frame) ----
    const float *gsrc = p.gsrc + (long long)plane * p.src_plane;
    const uint8_t *msrc = p.maps + (long long)plane * p.FH * p.FW;
    for (int y = warp; y < L.RH; y += NT / 32) {
        const int fy = fy0 + y;
        const bool yin = (unsigned)fy < (unsigned)p.FH;
        for (int x = lane; x < L.RW; x += 32) {
            const int fx = fx0 + x;
            float g = 0.f;
            int m = 0;
            if (yin && (unsigned)fx < (unsigned)p.FW) {
                m = msrc[(long long)fy * p.FW + fx];
                if (p.src_is_output) {  // the crop's transpose: grad_out inside, zero on the ring
                    const int oy = fy - p.R, ox = fx - p.R;
                    if ((unsigned)oy < (unsigned)p.H && (unsigned)ox < (unsigned)p.W)
                        g = gsrc[(long long)oy * p.src_pitch + ox];
                } else {
                    g = gsrc[(long long)fy * p.src_pitch + fx];
                }
            }
            gb[y * L.PG + x] = g;
            mb[y * L.PG + x] = (uint8_t)m;
        }
    }
    __syncthreads();

    // ---- pass V: per column, running up sums of c1..c6; F at output row y = s - 2R ----
    for (int c = threadIdx.x; c < L.RW; c += NT) {
        constexpr int P = R + 1;
        float2 r12[P], r34[P], r56[P];  // c-pairs by row slot (leave the window R + 1 rows later)
        float2 h13[P], h5e[P];          // (V1, V3)(s) and (V5, 0) by slot, plus (G5, G6) raw
        float2 e56[P];
        float2 V12 = make_float2(0.f, 0.f), V34 = V12, V56 = V12;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            r12[k] = make_float2(0.f, 0.f);
            r34[k] = r12[k];
            r56[k] = r12[k];
        }
        const int RH = L.RH;
        for (int s0 = 0; s0 < RH; s0 += P) {
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int s = s0 + k;
                if (s < RH) {
                    const int m = mb[s * L.PG + c];
                    const float w = gb[s * L.PG + c] * (m <= 4 ? iq : ih);
                    const unsigned cm = cmask(m);
                    const float2 n12 = make_float2((cm & 1u) ? w : 0.f, (cm & 2u) ? w : 0.f);
                    const float2 n34 = make_float2((cm & 4u) ? w : 0.f, (cm & 8u) ? w : 0.f);
                    const float2 n56 = make_float2((cm & 16u) ? w : 0.f, (cm & 32u) ? w : 0.f);
                    if (k == P - 1) {  // re-form the window sums from the ring (bounded FP32 drift)
                        r12[k] = n12;
                        r34[k] = n34;
                        r56[k] = n56;
                        V12 = r12[0];
                        V34 = r34[0];
                        V56 = r56[0];
#pragma unroll
                        for (int i = 1; i < P; ++i) {
                            V12 = __fadd2_rn(V12, r12[i]);
                            V34 = __fadd2_rn(V34, r34[i]);
                            V56 = __fadd2_rn(V56, r56[i]);
                        }
                    } else {
                        V12 = __fadd2_rn(V12, __fadd2_rn(n12, make_float2(-r12[k].x, -r12[k].y)));
                        V34 = __fadd2_rn(V34, __fadd2_rn(n34, make_float2(-r34[k].x, -r34[k].y)));
                        V56 = __fadd2_rn(V56, __fadd2_rn(n56, make_float2(-r56[k].x, -r56[k].y)));
                        r12[k] = n12;
                        r34[k] = n34;
                        r56[k] = n56;
                    }
                    h13[k] = make_float2(V12.x, V34.x);  // (V1, V3) at row s
                    h5e[k] = make_float2(V56.x, 0.f);    // V5 at row s
                    e56[k] = make_float2(m == 5 ? w : 0.f, m == 6 ? w : 0.f);
                    if (s >= 2 * R) {
                        const int sl = (k + 1) % P;  // row s - R
                        const int y = s - 2 * R;
                        const float f1 = h13[sl].x + V12.y - e56[sl].y;  // V1(y+R) + V2(y+2R) - G6(y+R)
                        const float f2 = h13[sl].y + V34.y - e56[sl].x;  // V3(y+R) + V4(y+2R) - G5(y+R)
                        const float f3 = h5e[sl].x + V56.y;              // V5(y+R) + V6(y+2R)
                        F12[y * L.PF + c] = make_float2(f1, f2);
                        F3[y * L.PG + c] = f3;
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---- pass H: g_in(y, x) = HL[F1](x) + HL[F2](x + R) - F3(x), x in [R, R + TW) ----
    float *gdst = p.gdst + (long long)plane * p.dst_plane;
    for (int item = warp; item < TW / SW; item += NT / 32) {
        const int y = lane;  // output row (TH == 32)
        const int xs = item * SW;
        constexpr int P = R + 1;
        constexpr int NS = SW + 2 * R;
        float2 r12[P], h12[P];
        float r3[P];
        float2 HL = make_float2(0.f, 0.f);
        const float2 *frow = F12 + y * L.PF + xs;
        const float *f3row = F3 + y * L.PG + xs;
        float *orow = gb + y * L.PG;  // the g box is dead after pass V: stage the tile there
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const int k = t % P;
            const float2 f = frow[t];
            r3[k] = f3row[t];
            if (t < R) {
                r12[k] = f;
                continue;
            }
            if (k == P - 1 || t == R || R <= 3) {
                r12[k] = f;
                HL = f;
#pragma unroll
                for (int i = 1; i <= R; ++i) HL = __fadd2_rn(HL, r12[(k + P - i) % P]);
            } else {  // slot k holds the value leaving the window (R + 1 steps back)
                HL = __fadd2_rn(HL, __fadd2_rn(f, make_float2(-r12[k].x, -r12[k].y)));
                r12[k] = f;
            }
            h12[k] = HL;
            if (t >= 2 * R) {
                const int sl = (k + 1) % P;   // column x = t - R (region coordinates)
                const int x = xs + t - 2 * R;  // tile column
                orow[x] = h12[sl].x + HL.y - r3[sl];
            }
        }
    }
    __syncthreads();
    // coalesced copy of the tile to the outgoing gradient frame
    for (int i = threadIdx.x; i < TH * TW; i += NT) {
        const int y = i / TW, x = i % TW;
        const int fy = ty0 + y, fx = tx0 + x;
        if (fy < p.FH && fx < p.FW) gdst[(long long)fy * p.dst_pitch + fx] = gb[y * L.PG + x];
    }
}

template <int R>
cudaError_t launch_bwd_tile(const BwdParams &p, dim3 grid, cudaStream_t s) {
    const BLayout L = make_blayout(R);
    cudaError_t e = cudaFuncSetAttribute(osbf_bwd_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes);
    if (e != cudaSuccess) return e;
    osbf_bwd_tile<R><<<grid, NT, L.bytes, s>>>(p);
    return cudaGetLastError();
}

}  // namespace bwd
}  // namespace osbf
