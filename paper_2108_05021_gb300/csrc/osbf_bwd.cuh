// osbf_bwd.cuh -- adjoint (backward) kernel of the One-Sided Box Filter (sm_103a).
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
//
// Organisation (persistent and TMA-fed, like the forward kernel):
//   * each CTA walks the tile list; a tile's region of the incoming gradient frame
//     (float32) and of the pass's selection map (uint8) arrive by two TMA tensor loads
//     on one mbarrier; out-of-frame elements read 0 (zero gradient; window 0 = none);
//   * pass V (one thread per region column) keeps the six column sums as three packed
//     f32x2 running sums over a register ring, and emits F1, F2 into a float2 field and
//     F3 in place over the gradient box (a thread overwrites only rows of its own column
//     that it has already consumed);
//   * pass H (one lane per tile row) keeps the two left row sums as one f32x2 and writes
//     g_in from registers into the outgoing gradient frame, four columns per 16-byte store;
//   * the tile grid is shifted by (16 - r % 16) % 16 columns, so both boxes start on
//     16 bytes (the TMA rule), and the stores are realigned in-lane.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "osbf_fwd2.cuh"

namespace osbf {
namespace bwd {

constexpr int TH = 32, TW = 128, SW = 32;
constexpr int NT = 160;  // one thread per region column (TW + 2r <= 160 for r <= 16)

struct BwdParams {
    float *gdst;          // outgoing gradient frame (pitch dst_pitch floats)
    long long dst_plane;  // floats per plane of gdst
    int dst_pitch;
    int FH, FW;
    int tiles_x, tiles_y, ntiles;
    int tx_shift;         // tile k starts at frame column k * TW - tx_shift
    unsigned int *err;    // device error word (bit 0: a bounded wait gave up)
};

struct BLayout {
    int RH, RW;  // region rows / columns
    int BXg;     // gradient box width (floats): >= RW + 3 (pass H's float4 over-read), BXg / 4 odd
    int BXm;     // selection box width (bytes): >= RW, a multiple of 16
    int PF;      // float2 row pitch of the (F1, F2) field: >= RW, PF % 4 == 2
    int off_g, off_m, off_f, bytes;
};

__host__ __device__ inline BLayout make_blayout(int R) {
    BLayout L;
    L.RH = TH + 2 * R;
    L.RW = TW + 2 * R;
    L.BXg = (L.RW + 3 + 3) / 4 * 4;
    if (((L.BXg / 4) & 1) == 0) L.BXg += 4;  // odd float4 pitch: conflict-free row-owner loads
    L.BXm = (L.RW + 15) / 16 * 16;
    L.PF = L.RW;
    while (L.PF % 4 != 2) ++L.PF;            // odd float4 pitch
    L.off_g = 0;
    L.off_m = v2::align128(L.RH * L.BXg * 4);
    L.off_f = v2::align128(L.off_m + L.RH * L.BXm);
    L.bytes = L.off_f + TH * L.PF * 8 + 16;  // + mbarrier
    return L;
}

// which column-sum inputs c1..c6 receive G_m (bit j-1 for c_j)
__device__ __forceinline__ unsigned cmask(int m) {
    // m:      1        2        3        4        5         6         7          8
    // c-bits: c3       c1       c2       c4       c3,c4     c1,c2     c1,c3,c5   c2,c4,c6
    const unsigned long long lut = (0x04ull << 8) | (0x01ull << 16) | (0x02ull << 24) | (0x08ull << 32) |
                                   (0x0Cull << 40) | (0x03ull << 48) | (0x15ull << 56);
    return m == 8 ? 0x2Au : (unsigned)(lut >> (8 * m)) & 0xFFu;
}

// pass V: thread = region column c.  Writes F1, F2 of tile rows y in [0, TH) to F12 and
// F3 over the gradient box's row y.
template <int R>
__device__ __forceinline__ void bwd_pass_v(float *__restrict__ gb, const uint8_t *__restrict__ mb,
                                           float2 *__restrict__ F12, const BLayout &L) {
    constexpr int P = R + 1;
    constexpr int RH = TH + 2 * R;
    constexpr float iq = 1.0f / float((R + 1) * (R + 1));
    constexpr float ih = 1.0f / float((R + 1) * (2 * R + 1));
    const int c = threadIdx.x;
    if (c >= L.RW) return;
    float *gcol = gb + c;
    const uint8_t *mcol = mb + c;
    float2 r12[P], r34[P], r56[P];  // (c1, c2), (c3, c4), (c5, c6) of the last P rows
    float2 q13[P];                  // (V1 - G6, V3 - G5) at each of the last P rows
    float q5[P];                    // V5 at each of the last P rows
#pragma unroll
    for (int k = 0; k < P; ++k) {
        r12[k] = make_float2(0.f, 0.f);
        r34[k] = r12[k];
        r56[k] = r12[k];
    }
    float2 V12 = make_float2(0.f, 0.f), V34 = V12, V56 = V12;
#pragma unroll
    for (int s = 0; s < RH; ++s) {
        const int k = s % P;
        const float gv = gcol[s * L.BXg];
        const int m = mcol[s * L.BXm];
        const float w = gv * (m <= 4 ? iq : ih);
        const unsigned cm = cmask(m);
        const float2 n12 = make_float2((cm & 1u) ? w : 0.f, (cm & 2u) ? w : 0.f);
        const float2 n34 = make_float2((cm & 4u) ? w : 0.f, (cm & 8u) ? w : 0.f);
        const float2 n56 = make_float2((cm & 16u) ? w : 0.f, (cm & 32u) ? w : 0.f);
        if (k == P - 1) {  // the ring holds the whole window: re-form the sums (bounded FP32 drift)
            r12[k] = n12;
            r34[k] = n34;
            r56[k] = n56;
            V12 = r12[0];
            V34 = r34[0];
            V56 = r56[0];
#pragma unroll
            for (int i = 1; i < P; ++i) {
                V12 = v2::add2(V12, r12[i]);
                V34 = v2::add2(V34, r34[i]);
                V56 = v2::add2(V56, r56[i]);
            }
        } else {  // slot k holds row s - R - 1 (zeros before the window fills)
            V12 = v2::add2(V12, v2::sub2(n12, r12[k]));
            V34 = v2::add2(V34, v2::sub2(n34, r34[k]));
            V56 = v2::add2(V56, v2::sub2(n56, r56[k]));
            r12[k] = n12;
            r34[k] = n34;
            r56[k] = n56;
        }
        // the parts of F1 / F2 / F3 that belong to row s as the upper window's bottom row
        q13[k] = make_float2(V12.x - (m == 6 ? w : 0.f), V34.x - (m == 5 ? w : 0.f));
        q5[k] = V56.x;
        if (s >= 2 * R) {
            const int y = s - 2 * R;
            const int sl = (s - R) % P;  // row s - R = y + R (frame row y of the formula)
            F12[y * L.PF + c] = make_float2(q13[sl].x + V12.y, q13[sl].y + V34.y);
            gcol[y * L.BXg] = q5[sl] + V56.y;  // row y of this column was consumed at step y
        }
    }
}

// pass H: lane = tile row, warp = one SW-column segment.  g_in of the tile goes from
// registers to the outgoing frame (SH realigns the 4-vectors to 16-byte columns), or --
// STAGE -- stays in `keep` (index = output column in the segment) for a staged write.
template <int R, bool STAGE>
__device__ __forceinline__ void bwd_pass_h(const float *__restrict__ gb, const float2 *__restrict__ F12,
                                           const BLayout &L, float *__restrict__ gdst, int pitch, int ty0, int tx0,
                                           int FH, int FW, float (&keep)[SW]) {
    constexpr int P = R + 1;
    constexpr int NS = SW + 2 * R;
    constexpr int SH = (4 - R % 4) % 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= TW / SW) return;
    const int y = lane, xs = warp * SW;
    const int fy = ty0 + y;
    const bool row_store = (unsigned)fy < (unsigned)FH;
    float *grow = gdst + (long long)(row_store ? fy : 0) * pitch + tx0 + xs;
    const float4 *frow = reinterpret_cast<const float4 *>(F12 + y * L.PF + xs);
    const float4 *f3row = reinterpret_cast<const float4 *>(gb + y * L.BXg + xs);
    float2 r12[P];
    float h1[P], r3[P];
#pragma unroll
    for (int k = 0; k < P; ++k) r12[k] = make_float2(0.f, 0.f);
    float2 HL = make_float2(0.f, 0.f);
    float4 v12 = make_float4(0.f, 0.f, 0.f, 0.f), v3 = v12;
    float o[4];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const int k = t % P;
        if ((t & 1) == 0) v12 = frow[t >> 1];
        if ((t & 3) == 0) v3 = f3row[t >> 2];
        const float2 f = (t & 1) ? make_float2(v12.z, v12.w) : make_float2(v12.x, v12.y);
        r3[k] = f4get(v3, t & 3);
        if (k == P - 1 || R <= 2) {
            r12[k] = f;
            HL = r12[0];
#pragma unroll
            for (int i = 1; i < P; ++i) HL = v2::add2(HL, r12[i]);
        } else {  // slot k holds column t - R - 1 (zeros before the window fills)
            HL = v2::add2(HL, v2::sub2(f, r12[k]));
            r12[k] = f;
        }
        h1[k] = HL.x;
        if (t >= 2 * R) {
            const int sl = (t - R) % P;  // region column t - R: the output pixel's column
            const int oo = t - 2 * R;    // output index within the segment
            const int slot = (oo - SH) & 3;
            o[slot] = h1[sl] + HL.y - r3[sl];
            if (STAGE) {
                keep[oo] = o[slot];
            } else if (SH > 0 && (oo < SH || oo >= SH + SW - 4)) {
                const int fx = tx0 + xs + oo;
                if (row_store && (unsigned)fx < (unsigned)FW) grow[oo] = o[slot];
            } else if (slot == 3) {
                const int fx = tx0 + xs + oo - 3;  // first column of the 4-vector (16-byte aligned)
                if (row_store && (unsigned)fx < (unsigned)FW)
                    *reinterpret_cast<float4 *>(grow + oo - 3) = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

// Staged stores (r <= 8): after the barrier that ends pass H, each pass-H warp parks its
// 32 x 32 results in the dead (F1, F2) field (rows of kStagePitch floats, an odd number of
// 16-byte chunks) and writes them row by row, a lane per column: 32 consecutive floats per
// store instruction instead of a 16-byte piece in each of 32 rows.  The 32 results a lane
// holds fit three CTAs per SM up to r = 4; at r = 5..8 the kernel runs two CTAs per SM
// with them (faster than three with per-lane stores: 193 -> 216 Gpixel/s at r = 5,
// 195 -> 205 at r = 8 on 4096^2 x 3).
constexpr int kStagePitch = 36;
template <int R> __host__ __device__ constexpr bool bwd_stage() { return R <= 8; }

template <int R>
__global__ void __launch_bounds__(NT, R <= 4 ? 3 : 2)
    osbf_bwd_kernel(const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap mmap,
                    const BwdParams p) {
    extern __shared__ __align__(128) unsigned char bsm[];
    const BLayout L = make_blayout(R);
    float *gb = reinterpret_cast<float *>(bsm + L.off_g);
    uint8_t *mb = bsm + L.off_m;
    float2 *F12 = reinterpret_cast<float2 *>(bsm + L.off_f);
    const uint32_t bar = v2::smem_u32(bsm + L.bytes - 16);
    const uint32_t box_bytes = (uint32_t)(L.RH * L.BXg * 4 + L.RH * L.BXm);
    const int tiles_per_plane = p.tiles_x * p.tiles_y;

    if (threadIdx.x == 0) {
        v2::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        v2::fence_proxy_async();
    }
    __syncthreads();

    auto origin = [&](int tile, int &plane, int &ty0, int &tx0) {
        plane = tile / tiles_per_plane;
        const int rem = tile % tiles_per_plane;
        ty0 = (rem / p.tiles_x) * TH;
        tx0 = (rem % p.tiles_x) * TW - p.tx_shift;
    };
    auto issue = [&](int tile) {
        int plane, ty0, tx0;
        origin(tile, plane, ty0, tx0);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(box_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(v2::smem_u32(gb)),
            "l"(reinterpret_cast<uint64_t>(&gmap)), "r"(tx0 - R), "r"(ty0 - R), "r"(plane), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(v2::smem_u32(mb)),
            "l"(reinterpret_cast<uint64_t>(&mmap)), "r"(tx0 - R), "r"(ty0 - R), "r"(plane), "r"(bar)
            : "memory");
    };
    auto warm = [&](int tile) {  // L2 prefetch one tile ahead of its shared-memory load
        int plane, ty0, tx0;
        origin(tile, plane, ty0, tx0);
        v2::tma_prefetch_l2_3d(&gmap, tx0 - R, ty0 - R, plane);
        v2::tma_prefetch_l2_3d(&mmap, tx0 - R, ty0 - R, plane);
    };

    int tile = blockIdx.x;
    if (tile < p.ntiles && threadIdx.x == 0) {
        issue(tile);
        if (tile + (int)gridDim.x < p.ntiles) warm(tile + gridDim.x);
    }
    uint32_t phase = 0;
    for (; tile < p.ntiles; tile += gridDim.x) {
        int plane, ty0, tx0;
        origin(tile, plane, ty0, tx0);
        const bool timed_out = !v2::mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(timed_out)) {
            // report; thread 0 gives the copies one more bounded wait, so the CTA's shared
            // memory outlives copies that are merely late
            if (threadIdx.x == 0) {
                atomicOr(p.err, 1u);
                v2::mbar_wait_bounded(bar, phase);
            }
            return;
        }
        phase ^= 1;
        bwd_pass_v<R>(gb, mb, F12, L);
        __syncthreads();
        float keep[SW];
        float *gplane = p.gdst + (long long)plane * p.dst_plane;
        bwd_pass_h<R, bwd_stage<R>()>(gb, F12, L, gplane, p.dst_pitch, ty0, tx0, p.FH, p.FW, keep);
        __syncthreads();
        if (bwd_stage<R>()) {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (warp < TW / SW) {
                float *stg = reinterpret_cast<float *>(F12) + warp * 32 * kStagePitch;
#pragma unroll
                for (int c = 0; c < SW / 4; ++c)
                    *reinterpret_cast<float4 *>(stg + lane * kStagePitch + 4 * c) =
                        make_float4(keep[4 * c], keep[4 * c + 1], keep[4 * c + 2], keep[4 * c + 3]);
                __syncwarp();
                const int fx = tx0 + warp * SW + lane;
                if ((unsigned)fx < (unsigned)p.FW) {
                    if (ty0 + TH <= p.FH) {  // the tile's rows all lie in the frame: no per-row checks
                        float *q = gplane + (long long)ty0 * p.dst_pitch + fx;
#pragma unroll
                        for (int j = 0; j < TH; ++j, q += p.dst_pitch) *q = stg[j * kStagePitch + lane];
                    } else {
                        for (int j = 0; j < TH; ++j)
                            if (ty0 + j < p.FH) gplane[(long long)(ty0 + j) * p.dst_pitch + fx] = stg[j * kStagePitch + lane];
                    }
                }
            }
            // the next tile's pass V writes (F1, F2) after the barrier at the top of the loop
        }
        const int next = tile + gridDim.x;
        if (next < p.ntiles && threadIdx.x == 0) {  // both boxes are dead: load the next tile
            v2::fence_proxy_async();
            issue(next);
            if (next + (int)gridDim.x < p.ntiles) warm(next + gridDim.x);
        }
    }
}

template <int R>
cudaError_t launch_bwd_kernel(const CUtensorMap &gmap, const CUtensorMap &mmap, const BwdParams &p, int grid,
                              cudaStream_t s) {
    const BLayout L = make_blayout(R);
    // staged results reuse the (F1, F2) field: TW / SW warps x 32 rows x kStagePitch floats
    if (bwd_stage<R>() && (size_t)TH * L.PF * 8 < (size_t)(TW / SW) * 32 * kStagePitch * 4) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(osbf_bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes);
    if (e != cudaSuccess) return e;
    osbf_bwd_kernel<R><<<grid, NT, L.bytes, s>>>(gmap, mmap, p);
    return cudaGetLastError();
}

template <int R>
int occupancy_bwd_kernel() {
    const BLayout L = make_blayout(R);
    if (cudaFuncSetAttribute(osbf_bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, osbf_bwd_kernel<R>, NT, L.bytes) != cudaSuccess) return 0;
    return n;
}

}  // namespace bwd
}  // namespace osbf
