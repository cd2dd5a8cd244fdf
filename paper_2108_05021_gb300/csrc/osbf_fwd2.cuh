// osbf_fwd2.cuh -- persistent, TMA-fed forward kernel of the One-Sided Box Filter (sm_103a).
//
// Same arithmetic as osbf_fwd.cuh (Eq. (6)-(13), the box kernels, Algorithm 2, the
// appendix's zero-outside-the-frame rule), organised for throughput:
//   * persistent CTAs walk the tile list; each tile's region (tile + halo) of the
//     source frame arrives by one TMA tensor load (out-of-frame elements are filled
//     with zeros by the copy engine, which is exactly the appendix's boundary), and
//     the next tile's load is issued as soon as the current input buffer is dead;
//   * pass V (one thread per column pair) keeps running column sums a(y) with packed
//     f32x2 instructions; pass H reads a(y) (up sum) and a(y + r) (down sum) of its row;
//   * pass H (one thread per row segment) keeps the left row sums (AL, BL) as a float2
//     and runs the window sums and scores with packed f32x2 instructions (two windows
//     per instruction); only the eight-way selection is scalar;
//   * single-pass launches write results from registers straight into the
//     destination frame, and the whole sweep of a segment is unrolled.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "osbf_fwd.cuh"

namespace osbf {
namespace v2 {

constexpr int TH = 32;   // tile rows
constexpr int TW = 128;  // tile columns
constexpr int SW = 32;   // pass-H segment width
constexpr int NT = 128;  // threads per CTA
constexpr unsigned long long kWaitNs = 1000000000ull;  // a tile load that has not landed in 1 s is an error

struct Layout2 {
    int EY, EX, RH0, RW0;
    int BX;      // TMA box width (elements) = row pitch of the input buffer
    int PU;      // float row pitch of U buffers (PU % 8 == 4: conflict-free row-owner float4 access)
    int P2;      // float row pitch of the column-sum field A
    int in_bytes;  // bytes of one TMA box
    int off_in, off_uf, off_ab, off_ua, off_ub, bytes;  // byte offsets (128-aligned)
    int off_st;  // tensor-store staging: NT/32 buffers of 32 x 32 floats, placed 1024-aligned at run time
    int off_ms;  // single-pass map staging: NT/32 buffers of 32 rows x kMapPitch bytes
    int off_xs;  // single-pass result staging: NT/32 buffers of 32 rows x kOutPitch floats
    int off_uc;  // EARLY: copy of the tile's TH centre rows of U^0 (row pitch PU), made by pass V
};

__host__ __device__ inline int align128(int b) { return (b + 127) & ~127; }

// direct: a single pass whose results go straight from registers to the destination
// frame (no U^1 buffer in shared memory)
// Row pitch (bytes) of a warp's map staging: 32 selections of a row plus the grid shift's
// offset, 9 words (odd: the row-owner word writes hit distinct banks)
constexpr int kMapPitch = 36;
// Row pitch (floats) of a warp's result staging (XSTAGE): 9 chunks of 16 bytes (odd: the
// row-owner 16-byte writes hit distinct banks)
constexpr int kOutPitch = 36;

template <typename T>
__host__ __device__ inline Layout2 make_layout2(int R, int D, bool direct = false, bool tstore = false,
                                                bool mstage = false, bool xstage = false, bool early = false) {
    Layout2 L;
    const int xa = 16 / (int)sizeof(T) < 4 ? 4 : 16 / (int)sizeof(T);
    L.EY = D * R;
    // direct kernels keep the halo at exactly R columns; the tile grid is shifted instead
    // (float32: by (4 - R % 4) % 4 columns, 16-bit: by (8 - R % 8) % 8), so the TMA box
    // still starts on 16 bytes
    L.EX = direct ? D * R : round_up(D * R, xa);
    L.RH0 = TH + 2 * L.EY;
    L.RW0 = TW + 2 * L.EX;
    // pass H sweeps full SW-wide segments over the widest output region (RW0 - 2R): the
    // last segment reads up to SW + 2R + 3 columns past its start
    const int xs_last = ((L.RW0 - 2 * R + SW - 1) / SW - 1) * SW;
    L.PU = xs_last + SW + 2 * R + 4;
    // fused passes also write intermediate rows up to 6 columns past the region; single-pass
    // (direct) kernels only read, up to column xs_last + SW + 2R + 3
    if (!direct && L.PU < L.RW0 + 8) L.PU = L.RW0 + 8;
    while (L.PU % 8 != 4) ++L.PU;
    L.P2 = L.PU;  // float row pitch of the column-sum field A (same conflict-free pitch)
    L.BX = sizeof(T) == 4 ? L.PU : round_up(L.PU, 8);
    L.in_bytes = L.BX * L.RH0 * (int)sizeof(T);
    const int rh1 = L.RH0 - 2 * R;  // rows of U^1 and of the (a, b) buffer
    int off = 0;
    L.off_in = off;
    off = align128(off + L.in_bytes);
    L.off_uf = off;  // float copy of the input (16-bit storage only)
    if (sizeof(T) != 4 && !early) off = align128(off + L.RH0 * L.PU * 4);

    L.off_ab = off;
    off = align128(off + (L.RH0 - R) * L.P2 * 4);
    L.off_ua = off;
    if (!direct) off = align128(off + rh1 * L.PU * 4);
    L.off_ub = off;
    if (D >= 2) off = align128(off + rh1 * L.PU * 4);
    L.off_st = off;
    if (tstore) off = align128(off + 1024 + (NT / 32) * 32 * 32 * 4);  // + slack to reach a 1024-byte boundary
    L.off_ms = off;
    if (mstage) off = align128(off + (NT / 32) * 32 * kMapPitch);
    L.off_xs = off;
    if (xstage) off = align128(off + (NT / 32) * 32 * kOutPitch * 4);
    L.off_uc = off;
    if (early) off = align128(off + TH * L.PU * 4);
    L.bytes = off + 16;  // + mbarrier
    return L;
}

struct Fwd2Params {
    void *dst;                 // frame (dst_is_output = 0) or the caller's output
    int dst_is_output;
    long long dst_plane;
    int dst_pitch;
    uint8_t *maps;             // selection maps [iters][P][FH][map_pitch] or null
    int map_pitch;             // bytes per map row (a multiple of 16)
    int map_iter0;
    long long map_iter_stride, map_plane;
    int H, W, FH, FW;
    int D;
    int tiles_x, tiles_y, ntiles;  // tile grid; ntiles = tiles_x * tiles_y * planes
    int ty_off, tx_off;
    int tx_shift;                  // tiles start at column k * TW - tx_shift (direct: float32 (4 - R % 4) % 4, 16-bit (8 - R % 8) % 8)
    int src_off;                   // PADIN: the source is the unpadded image, at frame coordinates - src_off (= r)
    int ty_shift;                  // tiles start at row k * TH - ty_shift
    unsigned int *err;         // device error word (bit 0: a bounded wait gave up)
};

// ----------------------------------------------------------------------------------
// TMA / mbarrier primitives (inline PTX)
// ----------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar,
                                            uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Pull a box of the tensor into L2 ahead of its load (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap *map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// Tensor store of a shared-memory box (bulk-group completion), and its waits.  The waits
// are hardware waits on this thread's own copies, not spin loops.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
// 32-byte store of eight floats (the address is 32-byte aligned)
__device__ __forceinline__ void st_global_v8(float *p, float4 a, float4 b) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for an mbarrier phase, giving up after kWaitNs (returns false then).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > kWaitNs) return false;
    }
}

// ----------------------------------------------------------------------------------
// packed f32x2 helpers
// ----------------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// four floats as four 16-bit storage values (round to nearest even), packed in 8 bytes
template <typename T> __device__ __forceinline__ uint2 pack4_16(float4 v);
template <> __device__ __forceinline__ uint2 pack4_16<__half>(float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
}
template <> __device__ __forceinline__ uint2 pack4_16<__nv_bfloat16>(float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
}
template <> __device__ __forceinline__ uint2 pack4_16<float>(float4) { return make_uint2(0u, 0u); }

// storage-type stores of four floats
template <typename T> __device__ __forceinline__ void cvt_store4(T *p, float4 v);
template <> __device__ __forceinline__ void cvt_store4<float>(float *p, float4 v) {
    *reinterpret_cast<float4 *>(p) = v;
}
template <> __device__ __forceinline__ void cvt_store4<__half>(__half *p, float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 w;
    w.x = *reinterpret_cast<uint32_t *>(&a);
    w.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = w;
}
template <> __device__ __forceinline__ void cvt_store4<__nv_bfloat16>(__nv_bfloat16 *p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 w;
    w.x = *reinterpret_cast<uint32_t *>(&a);
    w.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = w;
}

// ----------------------------------------------------------------------------------
// pass V on column pairs: a(y) = sum_{y-R..y} U(., x), stored at A[y - R] for region rows
// y in [R, RH).  NRH > 0: the row count is a compile-time constant (single-pass
// launches), so the sweep is fully unrolled.  UC (NRH > 0): the region's centre rows
// [R, R + TH) -- the pixels pass H filters -- are also copied to Uc (row pitch pc), so the
// input buffer is dead once pass V ends.
// ----------------------------------------------------------------------------------
// Two neighbouring source elements as floats (the pair starts on an even column).
template <typename TS> __device__ __forceinline__ float2 ld_pair(const TS *p);
template <> __device__ __forceinline__ float2 ld_pair<float>(const float *p) {
    return *reinterpret_cast<const float2 *>(p);
}
template <> __device__ __forceinline__ float2 ld_pair<__half>(const __half *p) {
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
template <> __device__ __forceinline__ float2 ld_pair<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}

// TS: the source's storage type (16-bit sources are widened in registers)
template <int R, int NRH, bool UC = false, typename TS = float>
__device__ __forceinline__ void pass_v2(const TS *__restrict__ U, int pu, float *__restrict__ A, int pa, int RH_rt,
                                        int RW, float *__restrict__ Uc = nullptr, int pc = 0) {
    static_assert(!UC || NRH > 0, "the centre-row copy: unrolled sweeps");
    constexpr int P = R + 1;
    const int npairs = (RW + 1) >> 1;
    for (int item = threadIdx.x; item < npairs; item += NT) {
        const int c = item * 2;
        const TS *col = U + c;
        float2 *acol = reinterpret_cast<float2 *>(A + c);
        float2 ring[P];
#pragma unroll
        for (int k = 0; k < P; ++k) ring[k] = make_float2(0.f, 0.f);
        float2 acc = make_float2(0.f, 0.f);
        // one row: slide the window sum by the row entering (v) and the one leaving
        // (ring[k]); once per ring period re-form it from the ring (bounded FP32 drift)
        auto update = [&](float2 v, int k) {
            if (k == P - 1) {
                ring[k] = v;
                acc = ring[0];
#pragma unroll
                for (int i = 1; i < P; ++i) acc = add2(acc, ring[i]);
            } else {
                acc = add2(acc, sub2(v, ring[k]));
                ring[k] = v;
            }
        };
        if (NRH > 0) {
            // loads run LA rows ahead in program order, so they never queue behind the
            // column-sum stores of earlier rows (the compiler cannot reorder them itself)
            constexpr int LA = 4;
            constexpr int NR = NRH > 0 ? NRH : 1;
            float2 q[LA];
#pragma unroll
            for (int i = 0; i < LA; ++i)
                q[i] = i < NR ? ld_pair<TS>(col + i * pu) : make_float2(0.f, 0.f);
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                const float2 v = q[s % LA];
                if (s + LA < NR) q[s % LA] = ld_pair<TS>(col + (s + LA) * pu);
                if (UC && s >= R && s < R + TH) *reinterpret_cast<float2 *>(Uc + (s - R) * pc + c) = v;
                update(v, s % P);
                if (s >= R) acol[(s - R) * (pa >> 1)] = acc;
            }
        } else {
            for (int s0 = 0; s0 < RH_rt; s0 += P) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int s = s0 + k;
                    if (s < RH_rt) {
                        update(ld_pair<TS>(col + s * pu), k);
                        if (s >= R) acol[(s - R) * (pa >> 1)] = acc;
                    }
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------------
// pass H: lane = row, warp = 32 rows x one SW-column segment
// ----------------------------------------------------------------------------------
struct Geom2 {
    int RHo, RWo;
    int fy0, fx0, FH, FW;
    int iy0, iy1, ix0, ix1;
    int oy, ox, ly, lx;  // DIRECT destination: frame offset of its origin and its extent
    int MP;              // map row pitch (bytes)
    int sx0, sy0, sz, sw, sh;  // TSTORE: destination coordinates of the tile's first output, plane, extent
};

template <int R, bool TIE_APP, bool IDX>
__device__ __forceinline__ void select2(float2 d41, float2 d32, float2 d56, float2 d87, float u, float &out, int &m) {
    // d_i for N1..N8
    const float dv[9] = {0.f, d41.y, d32.y, d32.x, d41.x, d56.x, d56.y, d87.y, d87.x};
    float d[8];
    int id[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        id[k] = tie_window<TIE_APP>(k);
        d[k] = dv[id[k]];
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

// 16-bit storage: the selection of select2, and the new value as the correctly rounded
// float32 quotient S_m / n_m of the selected window's sum, which the storage conversion
// then rounds once more.  For a mean lying exactly on a midpoint between two storage
// values that quotient is the midpoint itself and the conversion rounds it to even, as
// rounding the exact mean does; S_m * RN(1/n) alone can land an ulp to either side.
// The window sums ride through the tournament with their scores; the class of the
// winner (quadrant or half window) is decided by the last comparison.  The quotient
// comes from q = S * RN(1/n) and one correction step, q' = q + (S - q n) RN(1/n) with
// the residual exact in an FMA: Markstein's theorem (P. Markstein, IBM J. Res. Dev. 34,
// 1990) makes q' the correctly rounded S / n given a correctly rounded reciprocal and
// q within an ulp.
template <int R, bool TIE_APP, bool IDX>
__device__ __forceinline__ void select2_exact(float2 d41, float2 d32, float2 d56, float2 d87, float2 s41,
                                              float2 s32, float2 s56, float2 s87, float &out, int &m) {
    constexpr float nq = float((R + 1) * (R + 1)), nh = float((R + 1) * (2 * R + 1));
    constexpr float iq = 1.0f / nq, ih = 1.0f / nh;
    const float dv[9] = {0.f, d41.y, d32.y, d32.x, d41.x, d56.x, d56.y, d87.y, d87.x};
    const float sv[9] = {0.f, s41.y, s32.y, s32.x, s41.x, s56.x, s56.y, s87.y, s87.x};
    float d[8], sm[8];
    int id[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        id[k] = tie_window<TIE_APP>(k);
        d[k] = dv[id[k]];
        sm[k] = sv[id[k]];
    }
    auto pk = [&](int a, int b) {
        const bool take = fabsf(d[b]) < fabsf(d[a]);  // the lower tie position wins ties
        d[a] = take ? d[b] : d[a];
        sm[a] = take ? sm[b] : sm[a];
        if (IDX) id[a] = take ? id[b] : id[a];
    };
    pk(0, 1);
    pk(2, 3);
    pk(4, 5);
    pk(6, 7);
    pk(0, 2);
    pk(4, 6);
    const bool take = fabsf(d[4]) < fabsf(d[0]);
    const float S = take ? sm[4] : sm[0];
    m = take ? id[4] : id[0];
    // tie positions 0..3 hold the quadrants in the paper order, the half windows in the
    // appendix order
    const bool quad = TIE_APP ? take : !take;
    const float n = quad ? nq : nh, ri = quad ? iq : ih;
    const float q = S * ri;
    out = fmaf(fmaf(-q, n, S), ri, q);
}

// Output of pass H: a float buffer in shared memory (the next fused pass reads it), or
// -- DIRECT -- four results at a time straight into the destination frame in global
// memory (storage type T, 16- or 8-byte stores, rows and columns outside the frame skipped).
// FAST: the fast approximation (Sec. "Fast Approximation to One-sided Box Filter",
// Eq. (app)) -- the four quadrant sums are the same running sums, the half windows are
// the mean of two quadrant means, so the pixel row sums and the exact half sums go away.
// TSTORE (DIRECT float32, R % 4 == 0): each warp stages its 32 x 32 segment in a
// 1024-aligned shared buffer with the 128-byte swizzle (16-byte chunk c of row y at chunk
// c ^ (y & 7): the row-owner 4-vectors hit 8 distinct chunks per 8 lanes) and one lane
// writes it with a tensor store -- the copy engine writes whole lines instead of 32
// scattered 16-byte pieces per store instruction.
// STREAM (the streaming strip kernel, osbf_strip.cuh): the rows of a, b and U live in
// ring buffers; the caller passes this lane's row offsets (floats) sa, sb, su instead.
// V8 (DIRECT float32, R % 4 == 0, the destination's columns at the segment start on 32
// bytes): each lane writes its row's results eight at a time with one 32-byte store, an
// 8-column group whenever its first column lies inside the destination row (groups are
// aligned, so a destination whose width is a multiple of 8 -- or a frame, whose pitch
// padding is never read -- takes whole groups); no staging buffer.
template <int R, typename T, bool TIE_APP, bool MAPS, bool DIRECT, bool FAST = false, bool TSTORE = false,
          bool XSTAGE = false, bool STREAM = false, bool V8 = false>
__device__ __forceinline__ void pass_h2(const float *__restrict__ Uin, int pu_in, int urow0,
                                        const float *__restrict__ A, int pa, float *__restrict__ Uout, int pu_out,
                                        T *__restrict__ gdst, long long gpitch, const Geom2 &g,
                                        uint8_t *__restrict__ mplane, float *__restrict__ sbase = nullptr,
                                        const CUtensorMap *dmap = nullptr, uint8_t *__restrict__ mbase = nullptr,
                                        float *__restrict__ xbase = nullptr, int sa = 0, int sb = 0, int su = 0) {
    // XSTAGE (DIRECT float32): a warp's 32 x 32 results are staged like the selections
    // (float b of a row holds output b - MO) and written out row by row after the sweep, a
    // lane per column: 32 consecutive floats per store instruction instead of a 16-byte
    // piece in each of 32 rows, at any grid shift
    static_assert(!XSTAGE || (DIRECT && sizeof(T) == 4 && !TSTORE), "result staging: direct float32");
    static_assert(!V8 || (DIRECT && sizeof(T) == 4 && R % 4 == 0 && !TSTORE && !XSTAGE && !MAPS),
                  "32-byte stores: direct float32, R % 4 == 0, no maps");
    // DIRECT maps: a warp's 32 x 32 selections are staged (byte b of a row holds output
    // b - MO; MO puts every full 4-group of the shifted grid on a word) and written out row
    // by row after the sweep, one byte per lane: 32 contiguous bytes per store instruction
    // instead of one 4-byte piece in each of 32 rows
    constexpr int MO = DIRECT ? (4 - (4 - R % 4) % 4) % 4 : 0;
    constexpr int P = R + 1;         // ring period (the sweep is fully unrolled, so any period is static)
    constexpr int NS = SW + 2 * R;   // sweep steps of one segment (2R of warm-up)
    // tile grid shift mod 4 (both storage types: (4 - R % 4) % 4 = ((8 - R % 8) % 8) % 4)
    constexpr int SH = DIRECT ? (4 - R % 4) % 4 : 0;
    constexpr float iq = 1.0f / float((R + 1) * (R + 1));
    constexpr float ih = 1.0f / float((R + 1) * (2 * R + 1));
    const float2 iq2 = make_float2(iq, iq), ih2 = make_float2(ih, ih);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrb = (g.RHo + 31) >> 5;
    const int nseg = (g.RWo + SW - 1) / SW;
    for (int item = warp; item < nrb * nseg; item += NT / 32) {
        const int rbk = item % nrb, seg = item / nrb;
        const int yo = rbk * 32 + lane;
        float *sbuf = TSTORE ? sbase + warp * 32 * 32 : nullptr;
        uint8_t *mst = (MAPS && DIRECT) ? mbase + warp * 32 * kMapPitch : nullptr;
        float *xst = XSTAGE ? xbase + warp * 32 * kOutPitch : nullptr;
        if (TSTORE) {
            if (lane == 0) bulk_wait_read_all();  // the previous tensor store has read this buffer
            __syncwarp();
        }
        const bool row_ok = yo < g.RHo;
        const int yr = row_ok ? yo : g.RHo - 1;
        const int xs = seg * SW;
        // a: up column sums, b: down column sums
        const float4 *arow = reinterpret_cast<const float4 *>(A + (STREAM ? sa : yr * pa) + xs);
        const float4 *brow = reinterpret_cast<const float4 *>(A + (STREAM ? sb : (yr + R) * pa) + xs);
        const float4 *urow = reinterpret_cast<const float4 *>(Uin + (STREAM ? su : (yr + urow0) * pu_in) + xs);
        float4 *orow = reinterpret_cast<float4 *>(Uout + yr * pu_out + xs);
        const int fy = g.fy0 + yo;
        // DIRECT: frame row fy lands in row fy - g.oy of the destination (0 for a frame,
        // r for the cropped output), which has g.ly rows and g.lx columns
        const int dy = fy - g.oy;
        const bool row_store = DIRECT ? (row_ok && (unsigned)dy < (unsigned)g.ly) : row_ok;
        T *grow = DIRECT ? gdst + (long long)(row_store ? dy : 0) * gpitch + (g.fx0 - g.ox) + xs : nullptr;
        const bool row_map =
            MAPS && mplane != nullptr && row_ok && (unsigned)fy < (unsigned)g.FH && yo >= g.iy0 && yo < g.iy1;
        float ra[P], rb[P], ru[P], h6[P];  // raw a, b, U; and N6 sums (N5 at x is N6 at x - r)
        float2 hab[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            ra[k] = 0.f;
            rb[k] = 0.f;
            ru[k] = 0.f;
        }
        float2 ABL = make_float2(0.f, 0.f);  // (AL, BL): left row sums of a and b
        float UL = 0.f;
        // loads run one 4-column group ahead in program order (ahead of this group's stores)
        constexpr int NG = (NS + 3) / 4;
        float4 va = arow[0], vb = brow[0], vu = urow[0];
        float4 na = va, nb = vb, nu4 = vu;
        float o[4];
        uint2 held = make_uint2(0u, 0u);  // 16-bit DIRECT frames: the first half of a 16-byte store
        float4 held8 = make_float4(0.f, 0.f, 0.f, 0.f);  // V8: the first half of a 32-byte store
        uint32_t mw = 0;  // DIRECT maps: selections of the current 4-column group
        // the whole segment is unrolled: ring slots, loads, warm-up and stores are static
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const int k = t % P;
            if ((t & 3) == 0) {
                va = na;
                vb = nb;
                vu = nu4;
                if ((t >> 2) + 1 < NG) {
                    na = arow[(t >> 2) + 1];
                    nb = brow[(t >> 2) + 1];
                    nu4 = urow[(t >> 2) + 1];
                }
            }
            const float a = f4get(va, t & 3), b = f4get(vb, t & 3), u = f4get(vu, t & 3);
            if (t < R) {
                // warm-up: no window is complete yet; only fill the rings
                ra[k] = a;
                rb[k] = b;
                ru[k] = u;
                continue;
            }
            if (R <= 3 || k == P - 1 || t == R) {
                // direct sum over the ring's last R+1 entries (cheap for small r; resets
                // the running sums' FP32 drift once per ring period for large r)
                ra[k] = a;
                rb[k] = b;
                ru[k] = u;
                float al = a, bl = b, ul = u;
#pragma unroll
                for (int i = 1; i <= R; ++i) {
                    al += ra[(k + P - i) % P];
                    bl += rb[(k + P - i) % P];
                    if (!FAST) ul += ru[(k + P - i) % P];
                }
                ABL = make_float2(al, bl);
                if (!FAST) UL = ul;
            } else {
                const int so = (k + 2 * P - R - 1) % P;  // the value leaving the window
                ABL = make_float2(ABL.x + (a - ra[so]), ABL.y + (b - rb[so]));
                if (!FAST) UL += u - ru[so];
                ra[k] = a;
                rb[k] = b;
                ru[k] = u;
            }
            hab[k] = ABL;
            // N6 at the current column: the right half window of column x = t - R
            const float n6 = FAST ? 0.f : (ABL.x + ABL.y) - UL;
            if (!FAST) h6[k] = n6;
            if (t >= 2 * R) {
                const int sl = (k + P - R) % P;  // column x = t - R; (AL, BL) at x+R is current
                const float2 ABx = hab[sl];      // (AL(x), BL(x)) = (N4, N1)
                const float ux = ru[sl];
                const float2 nu = make_float2(-ux, -ux);
                const float2 d41 = fma2(ABx, iq2, nu);
                const float2 d32 = fma2(ABL, iq2, nu);  // (N3, N2) = (AL(x+r), BL(x+r))
                float2 d56, d87;
                float2 s56 = make_float2(0.f, 0.f), s87 = s56;  // (N5, N6) and (N8, N7) sums
                if (FAST) {
                    // Eq. (app): d5 = (d4 + d1)/2, d6 = (d3 + d2)/2, d8 = (d4 + d3)/2, d7 = (d1 + d2)/2
                    const float2 h = make_float2(0.5f, 0.5f);
                    d56 = mul2(add2(make_float2(d41.x, d32.x), make_float2(d41.y, d32.y)), h);
                    d87 = mul2(add2(d41, d32), h);
                } else {
                    const float2 sum = add2(ABx, ABL);
                    s87 = make_float2(sum.x - ra[sl], sum.y - rb[sl]);  // (N8, N7)
                    s56 = make_float2(h6[sl], n6);                      // N5(x) = N6(x - r) : left half of x
                    d56 = fma2(s56, ih2, nu);
                    d87 = fma2(s87, ih2, nu);
                }
                float outv;
                int m;
                if constexpr (sizeof(T) == 2 && !FAST) {
                    select2_exact<R, TIE_APP, MAPS>(d41, d32, d56, d87, ABx, ABL, s56, s87, outv, m);
                } else {
                    select2<R, TIE_APP, MAPS>(d41, d32, d56, d87, ux, outv, m);
                }
                const int xo = xs + t - 2 * R;
                const int oo = t - 2 * R;  // output index within the segment
                // column of output oo is congruent to oo - SH mod 4 (SH: the grid shift)
                const int slot = (oo - SH) & 3;
                o[slot] = storage_round<T>(outv);
                if (MAPS && DIRECT) {  // four selections per 32-bit word, like the outputs
                    mw = slot == 0 ? (uint32_t)m : mw | ((uint32_t)m << (8 * slot));
                } else if (MAPS) {
                    const int fx = g.fx0 + xo;
                    if (row_map && (unsigned)fx < (unsigned)g.FW && xo >= g.ix0 && xo < g.ix1)
                        mplane[(long long)fy * g.MP + fx] = (uint8_t)m;
                }
                if (DIRECT && SH > 0 && (oo < SH || oo >= SH + SW - 4)) {
                    // the segment's first SH and last 4 - SH outputs share a 4-vector with a
                    // neighbouring segment: store them one by one
                    const int dx = g.fx0 - g.ox + xo;
                    if (XSTAGE)
                        xst[lane * kOutPitch + oo + MO] = o[slot];
                    else if (row_store && (unsigned)dx < (unsigned)g.lx)
                        grow[oo] = from_f<T>(o[slot]);
                    if (MAPS) mst[lane * kMapPitch + oo + MO] = (uint8_t)m;
                } else if (slot == 3) {
                    const float4 v = make_float4(o[0], o[1], o[2], o[3]);
                    if (TSTORE) {
                        const int c = (oo - 3) >> 2;  // 16-byte chunk of the staged row
                        *reinterpret_cast<float4 *>(sbuf + lane * 32 + ((c ^ (lane & 7)) << 2)) = v;
                    } else if (DIRECT) {
                        const int dx = g.fx0 - g.ox + xo - 3;  // first column of the 4-vector
                        if constexpr (sizeof(T) == 2) {
                            // 16-bit frames: frame columns 8k..8k+7 leave as one 16-byte store
                            // when both 4-vectors are this segment's; the tile origin is
                            // -(8 - R % 8) % 8 mod 8, so each vector's half is static
                            constexpr int SH8 = (8 - R % 8) % 8;
                            // (static once the sweep is unrolled)
                            const int half = (oo - 3 - SH8) & 7;  // 0: columns 8k.., 4: 8k+4..
                            const bool lo_full = oo - 4 >= 3 && !(SH > 0 && (oo - 4 < SH || oo - 4 >= SH + SW - 4));
                            const bool hi_full = oo + 4 < SW && !(SH > 0 && (oo + 4 < SH || oo + 4 >= SH + SW - 4));
                            const bool pairs = g.oy == 0 && (gpitch & 7) == 0;  // a frame, rows on 16 bytes
                            if (pairs && half == 0 && hi_full) {
                                held = pack4_16<T>(v);  // stored with its partner
                            } else if (pairs && half == 4 && lo_full) {
                                if (row_store && (unsigned)(dx - 4) < (unsigned)g.lx) {
                                    const uint2 w = pack4_16<T>(v);
                                    *reinterpret_cast<uint4 *>(grow + (oo - 7)) = make_uint4(held.x, held.y, w.x, w.y);
                                }
                            } else if (row_store && (unsigned)dx < (unsigned)g.lx) {
                                cvt_store4<T>(grow + (oo - 3), v);
                            }
                        } else if (XSTAGE) {
                            *reinterpret_cast<float4 *>(xst + lane * kOutPitch + oo - 3 + MO) = v;
                        } else if (V8) {
                            if ((oo & 7) == 3) {
                                held8 = v;
                            } else if (row_store && (unsigned)(dx - 4) < (unsigned)g.lx) {
                                st_global_v8(grow + (oo - 7), held8, v);
                            }
                        } else if (row_store && (unsigned)dx < (unsigned)g.lx) {
                            cvt_store4<T>(grow + (oo - 3), v);
                        }
                        if (MAPS) *reinterpret_cast<uint32_t *>(mst + lane * kMapPitch + oo - 3 + MO) = mw;
                    } else if (row_ok) {
                        orow[oo >> 2] = v;
                    }
                }
            }
        }
        if (XSTAGE) {
            __syncwarp();
            const int dx = g.fx0 - g.ox + xs + lane;  // this lane's destination column
            if ((unsigned)dx < (unsigned)g.lx) {
                const int dy0 = g.fy0 - g.oy + rbk * 32;
                const int nr = g.RHo - rbk * 32 < 32 ? g.RHo - rbk * 32 : 32;
                const float *src = xst + lane + MO;
                if (nr == 32 && dy0 >= 0 && dy0 + 32 <= g.ly) {
                    // every row of the segment lies inside the destination: no per-row checks
                    T *q = gdst + (long long)dy0 * gpitch + dx;
#pragma unroll
                    for (int j = 0; j < 32; ++j, q += gpitch) *q = from_f<T>(src[j * kOutPitch]);
                } else {
                    for (int j = 0; j < nr; ++j)
                        if ((unsigned)(dy0 + j) < (unsigned)g.ly)
                            gdst[(long long)(dy0 + j) * gpitch + dx] = from_f<T>(src[j * kOutPitch]);
                }
            }
            __syncwarp();  // the next segment reuses the buffer
        }
        if (MAPS && DIRECT) {
            __syncwarp();
            const int fx = g.fx0 + xs + lane;  // this lane's frame column
            if (mplane != nullptr && (unsigned)fx < (unsigned)g.FW) {
                const int fy0 = g.fy0 + rbk * 32;
                const int nr = g.RHo - rbk * 32 < 32 ? g.RHo - rbk * 32 : 32;
                const uint8_t *src = mst + lane + MO;
                if (nr == 32 && fy0 >= 0 && fy0 + 32 <= g.FH) {
                    uint8_t *q = mplane + (long long)fy0 * g.MP + fx;
#pragma unroll
                    for (int j = 0; j < 32; ++j, q += g.MP) *q = src[j * kMapPitch];
                } else {
                    for (int j = 0; j < nr; ++j)
                        if ((unsigned)(fy0 + j) < (unsigned)g.FH)
                            mplane[(long long)(fy0 + j) * g.MP + fx] = src[j * kMapPitch];
                }
            }
            __syncwarp();  // the next segment reuses the buffer
        }
        if (TSTORE) {
            // every lane's staged writes become visible to the copy engine, then one lane
            // stores the segment (rows and columns past the destination are clipped by it)
            fence_proxy_async();
            __syncwarp();
            const int x = g.sx0 + xs, y = g.sy0 + rbk * 32;
            if (lane == 0 && x < g.sw && y < g.sh) {
                tma_store_3d(dmap, smem_u32(sbuf), x, y, g.sz);
                bulk_commit();
            }
        }
    }
}

// Zero the cells of a fused intermediate region that lie outside the padded frame (the
// next pass must read zeros there, as the appendix's convolution does).
__device__ __forceinline__ void zero_outside(float *__restrict__ U, int pu, int RHo, int RWo, int fy0, int fx0, int FH,
                                             int FW) {
    for (int i = threadIdx.x; i < RHo * RWo; i += NT) {
        const int y = i / RWo, x = i % RWo;
        if ((unsigned)(fy0 + y) >= (unsigned)FH || (unsigned)(fx0 + x) >= (unsigned)FW) U[y * pu + x] = 0.f;
    }
}

// ----------------------------------------------------------------------------------
// the persistent kernel
// ----------------------------------------------------------------------------------
// Tile order: plane by plane, row by row.
__device__ __forceinline__ void tile_origin(const Fwd2Params &p, int tile, int &plane, int &ty0, int &tx0) {
    const int per = p.tiles_x * p.tiles_y;
    plane = tile / per;
    const int rem = tile - plane * per;
    ty0 = (rem / p.tiles_x + p.ty_off) * TH - p.ty_shift;
    tx0 = (rem % p.tiles_x + p.tx_off) * TW - p.tx_shift;
}

// DIRECT: one pass per launch whose results (and selections, with MAPS) go from
// registers straight into the destination (D == 1, halo EX == R); otherwise every pass
// lands in shared memory and the tile interior is copied out at the end.
// PADIN (first pass): the source tensor map is the unpadded image; the copy engine fills
// zeros beyond it, and tiles touching its border then set every frame cell outside the
// image to its nearest image cell (the appendix's replicate pad), which always lies in
// the same box -- no separate padding pass.
// EARLY (single passes without maps: float32 frame to frame at R % 4 == 0, 16-bit storage
// at any R): pass V copies the centre rows that pass H reads (16-bit sources widened in
// registers, so no float copy of the whole box is made), and the next tile's load is
// issued before pass H instead of after it and lands while pass H runs.  Float32 results
// leave by 32-byte register stores (the frame's columns at a segment start lie on 32
// bytes: no grid shift, a 32-float row pitch), which frees the tensor-store staging for
// the copy; 16-bit results by the 16-byte register stores of the other 16-bit kernels.
template <typename T, int R, bool TIE_APP, bool MAPS, bool DIRECT, bool FAST = false, bool TSTORE = false,
          bool XSTAGE = false, bool PADIN = false, bool EARLY = false>
__global__ void __launch_bounds__(NT, DIRECT ? (R <= 9 && !MAPS && !TSTORE && !XSTAGE &&
                                                !(EARLY && sizeof(T) == 4) ? 4 : 3)
                                             : 2)
    osbf_fwd2(const __grid_constant__ CUtensorMap src, const __grid_constant__ CUtensorMap dmap, const Fwd2Params p) {
    static_assert(!TSTORE || (DIRECT && sizeof(T) == 4 && !MAPS && R % 4 == 0), "tensor stores: float32, R % 4 == 0");
    static_assert(!PADIN || TSTORE, "the padding first pass: the tensor-store kernel");
    static_assert(!EARLY || (DIRECT && !MAPS && !TSTORE && !XSTAGE && (sizeof(T) != 4 || R % 4 == 0)),
                  "early loads: single passes without maps (float32: R % 4 == 0)");
    extern __shared__ __align__(128) unsigned char smem2[];
    const int D = DIRECT ? 1 : p.D;  // single-pass kernels: the whole layout is a compile-time constant
    const Layout2 L = make_layout2<T>(R, D, DIRECT, TSTORE, MAPS && DIRECT, XSTAGE, EARLY);
    float *sbase = nullptr;  // TSTORE staging, 1024-aligned (the 128-byte swizzle repeats every 1024 bytes)
    if (TSTORE) {
        const uint32_t a = smem_u32(smem2 + L.off_st);
        sbase = reinterpret_cast<float *>(smem2 + L.off_st + (((a + 1023u) & ~1023u) - a));
    }
    T *bin = reinterpret_cast<T *>(smem2 + L.off_in);
    float *uf = reinterpret_cast<float *>(smem2 + (sizeof(T) == 4 ? L.off_in : L.off_uf));
    float *A = reinterpret_cast<float *>(smem2 + L.off_ab);
    float *Ua = reinterpret_cast<float *>(smem2 + L.off_ua);
    float *Ub = reinterpret_cast<float *>(smem2 + L.off_ub);
    const uint32_t bar = smem_u32(smem2 + L.bytes - 16);
    const int pu0 = sizeof(T) == 4 ? L.BX : L.PU;  // pitch of U^0 as a float buffer

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();

    auto issue = [&](int tile) {
        int plane, ty0, tx0;
        tile_origin(p, tile, plane, ty0, tx0);
        const int so = PADIN ? p.src_off : 0;
        tma_load_3d(smem_u32(bin), &src, tx0 - L.EX - so, ty0 - L.EY - so, plane, bar, (uint32_t)L.in_bytes);
    };
    // L2 prefetch of a tile's box: issued one tile ahead of its shared-memory load, so
    // that load is served from L2 instead of DRAM
    auto warm = [&](int tile) {
        int plane, ty0, tx0;
        tile_origin(p, tile, plane, ty0, tx0);
        const int so = PADIN ? p.src_off : 0;
        tma_prefetch_l2_3d(&src, tx0 - L.EX - so, ty0 - L.EY - so, plane);
    };
    auto prefetch = [&](int tile) {
        const int next = tile + gridDim.x;
        if (next < p.ntiles && threadIdx.x == 0) {
            fence_proxy_async();
            issue(next);
            if (next + (int)gridDim.x < p.ntiles) warm(next + gridDim.x);
        }
    };

    int tile = blockIdx.x;
    if (tile < p.ntiles && threadIdx.x == 0) {
        issue(tile);
        if (tile + (int)gridDim.x < p.ntiles) warm(tile + gridDim.x);
    }
    uint32_t phase = 0;
    for (; tile < p.ntiles; tile += gridDim.x) {
        int plane, ty0, tx0;
        tile_origin(p, tile, plane, ty0, tx0);
        // wait for this tile's region (bounded: a copy that never lands is reported, not waited on forever)
        const bool timed_out = !mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(timed_out)) {
            // report; thread 0 gives the copy one more bounded wait, so the CTA's shared
            // memory outlives a copy that is merely late
            if (threadIdx.x == 0) {
                atomicOr(p.err, 1u);
                mbar_wait_bounded(bar, phase);
            }
            if (TSTORE && (threadIdx.x & 31) == 0) bulk_wait_all();
            return;
        }
        phase ^= 1;
        if (PADIN) {
            // frame coordinates of the box origin; the image occupies [R, R+H) x [R, R+W)
            const int by0 = ty0 - L.EY, bx0 = tx0 - L.EX;
            if (by0 < R || by0 + L.RH0 > R + p.H || bx0 < R || bx0 + L.BX > R + p.W) {
                float *ub = reinterpret_cast<float *>(bin);
                // box rows and columns of the image and of the frame
                const int iy0 = max(R - by0, 0), iy1 = min(R + p.H - by0, L.RH0);
                const int ix0 = max(R - bx0, 0), ix1 = min(R + p.W - bx0, L.BX);
                const int fy0 = max(-by0, 0), fy1 = min(p.FH - by0, L.RH0);
                const int fx0 = max(-bx0, 0), fx1 = min(p.FW - bx0, L.BX);
                // 1. image rows: the left and right frame-ring columns copy the image's edge column
                const int nl = ix0 - fx0, nr = fx1 - ix1, ncol = nl + nr;
                for (int i = threadIdx.x; i < (iy1 - iy0) * ncol; i += NT) {
                    const int y = iy0 + i / ncol, k = i % ncol;
                    const int x = k < nl ? fx0 + k : ix1 + (k - nl);
                    ub[y * L.BX + x] = ub[y * L.BX + (k < nl ? ix0 : ix1 - 1)];
                }
                __syncthreads();
                // 2. frame-ring rows above and below the image copy its edge row (now complete)
                const int nt = iy0 - fy0, nb = fy1 - iy1, nrow = nt + nb, w = fx1 - fx0;
                for (int i = threadIdx.x; i < nrow * w; i += NT) {
                    const int k = i / w, x = fx0 + i % w;
                    const int y = k < nt ? fy0 + k : iy1 + (k - nt);
                    ub[y * L.BX + x] = ub[(k < nt ? iy0 : iy1 - 1) * L.BX + x];
                }
                __syncthreads();
            }
        }

        bool prefetched = false;
        if (sizeof(T) != 4 && !EARLY) {  // widen the 16-bit box into the float buffer, then the box is free
            const int w4 = (L.PU - 4) / 4;
            for (int i = threadIdx.x; i < L.RH0 * w4; i += NT) {
                const int y = i / w4, x = (i % w4) * 4;
                const T *q = bin + y * L.BX + x;
                *reinterpret_cast<float4 *>(uf + y * L.PU + x) =
                    make_float4(to_f(q[0]), to_f(q[1]), to_f(q[2]), to_f(q[3]));
            }
            __syncthreads();
            prefetch(tile);
            prefetched = true;
        }
        const bool interior = ty0 - L.EY >= 0 && tx0 - L.EX >= 0 && ty0 + TH + L.EY <= p.FH &&
                              tx0 + TW + L.EX <= p.FW;
        T *gdst = reinterpret_cast<T *>(p.dst) + (long long)plane * p.dst_plane;
        for (int j = 1; j <= D; ++j) {
            const float *Uin = j == 1 ? uf : ((j & 1) ? Ub : Ua);
            const int puin = j == 1 ? pu0 : L.PU;
            float *Uout = (j & 1) ? Ua : Ub;
            const int RH = L.RH0 - 2 * (j - 1) * R, RW = L.RW0 - 2 * (j - 1) * R;
            float *Uc = reinterpret_cast<float *>(smem2 + L.off_uc);
            if (EARLY) {
                pass_v2<R, TH + 2 * R, true, T>(bin, L.BX, A, L.P2, RH, RW, Uc, L.PU);
                __syncthreads();
                prefetch(tile);  // the input box is dead: its next load overlaps pass H
                prefetched = true;
            } else if (DIRECT) {
                pass_v2<R, TH + 2 * R>(Uin, puin, A, L.P2, RH, RW);
                __syncthreads();
            } else {
                pass_v2<R, 0>(Uin, puin, A, L.P2, RH, RW);
                __syncthreads();
            }
            Geom2 g;
            g.RHo = RH - 2 * R;
            g.RWo = RW - 2 * R;
            g.fy0 = ty0 - (L.EY - j * R);
            g.fx0 = tx0 - (L.EX - j * R);
            g.FH = p.FH;
            g.FW = p.FW;
            g.iy0 = L.EY - j * R;
            g.iy1 = g.iy0 + TH;
            g.ix0 = L.EX - j * R;
            g.ix1 = g.ix0 + TW;
            g.oy = p.dst_is_output ? R : 0;  // DIRECT into the cropped output needs W % 4 == 0
            g.ox = g.oy;
            g.ly = p.dst_is_output ? p.H : p.FH;
            g.lx = p.dst_is_output ? p.W : p.FW;
            g.MP = p.map_pitch;
            if (TSTORE) {  // destination coordinates of the tile's first output column / row
                g.sx0 = g.fx0 - g.ox;
                g.sy0 = g.fy0 - g.oy;
                g.sz = plane;
                g.sw = g.lx;
                g.sh = g.ly;
            }
            uint8_t *mplane = nullptr;
            if (MAPS && p.maps)
                mplane =
                    p.maps + (long long)(p.map_iter0 + j - 1) * p.map_iter_stride + (long long)plane * p.map_plane;
            pass_h2<R, T, TIE_APP, MAPS, DIRECT, FAST, TSTORE, XSTAGE, false, EARLY && sizeof(T) == 4>(
                EARLY ? Uc : Uin, EARLY ? L.PU : puin, EARLY ? 0 : R, A, L.P2, Uout, L.PU, gdst, p.dst_pitch, g,
                mplane, sbase, &dmap, smem2 + L.off_ms, reinterpret_cast<float *>(smem2 + L.off_xs));
            // single passes whose next load is already out (EARLY, and 16-bit storage, whose
            // box is widened and freed before pass V): the barrier after the next tile's load
            // wait orders this pass H's reads before the next tile's shared-memory writes
            if (!(DIRECT && (EARLY || sizeof(T) != 4))) __syncthreads();
            if (!prefetched) {  // float32: U^0 lived in the TMA box; it is dead after pass 1
                prefetch(tile);
                prefetched = true;
            }
            if (!DIRECT && j < D && !interior) {
                zero_outside(Uout, L.PU, g.RHo, g.RWo, g.fy0, g.fx0, p.FH, p.FW);
                __syncthreads();
            }
        }
        if (DIRECT) continue;  // results already in the destination frame

        // store the tile interior of U^D (row-wise, coalesced)
        const float *UD = (D & 1) ? Ua : Ub;
        const int cx = L.EX - D * R;
        if (!p.dst_is_output) {
            if ((cx & 3) == 0) {
                for (int i = threadIdx.x; i < TH * (TW / 4); i += NT) {
                    const int y = i / (TW / 4), x = (i % (TW / 4)) * 4;
                    const int fy = ty0 + y, fx = tx0 + x;
                    if (fy < p.FH && fx < p.FW)
                        cvt_store4<T>(gdst + (long long)fy * p.dst_pitch + fx,
                                      *reinterpret_cast<const float4 *>(UD + y * L.PU + cx + x));
                }
            } else {
                for (int i = threadIdx.x; i < TH * TW; i += NT) {
                    const int y = i / TW, x = i % TW;
                    const int fy = ty0 + y, fx = tx0 + x;
                    if (fy < p.FH && fx < p.FW) gdst[(long long)fy * p.dst_pitch + fx] = from_f<T>(UD[y * L.PU + cx + x]);
                }
            }
        } else {
            for (int i = threadIdx.x; i < TH * TW; i += NT) {
                const int y = i / TW, x = i % TW;
                const int oy = ty0 + y - R, ox = tx0 + x - R;
                if (oy >= 0 && oy < p.H && ox >= 0 && ox < p.W)
                    gdst[(long long)oy * p.dst_pitch + ox] = from_f<T>(UD[y * L.PU + cx + x]);
            }
        }
        __syncthreads();
    }
    if (TSTORE && (threadIdx.x & 31) == 0) bulk_wait_all();  // this warp's last segment store is complete
}

// dmap: the destination's tensor map (read only by TSTORE kernels; any map otherwise)
template <typename T, int R, bool TIE_APP, bool MAPS, bool DIRECT, bool FAST = false, bool TSTORE = false,
          bool XSTAGE = false, bool PADIN = false, bool EARLY = false>
cudaError_t launch_fwd2(const CUtensorMap &src, const Fwd2Params &p, int grid, cudaStream_t stream,
                        const CUtensorMap *dmap = nullptr) {
    const Layout2 L = make_layout2<T>(R, p.D, DIRECT, TSTORE, MAPS && DIRECT, XSTAGE, EARLY);
    auto kern = osbf_fwd2<T, R, TIE_APP, MAPS, DIRECT, FAST, TSTORE, XSTAGE, PADIN, EARLY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, L.bytes, stream>>>(src, dmap ? *dmap : src, p);
    return cudaGetLastError();
}

template <typename T, int R, bool TIE_APP, bool MAPS, bool DIRECT, bool FAST = false, bool TSTORE = false,
          bool XSTAGE = false, bool EARLY = false>
int occupancy_fwd2(int D) {
    const Layout2 L = make_layout2<T>(R, D, DIRECT, TSTORE, MAPS && DIRECT, XSTAGE, EARLY);
    auto kern = osbf_fwd2<T, R, TIE_APP, MAPS, DIRECT, FAST, TSTORE, XSTAGE, false, EARLY>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT, L.bytes) != cudaSuccess) return 0;
    return n;
}

}  // namespace v2
}  // namespace osbf
