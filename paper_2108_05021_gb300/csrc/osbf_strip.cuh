// osbf_strip.cuh -- streaming strip forward kernel of the One-Sided Box Filter (sm_103a).
//
// One pass per launch, float32 storage, paper tie order, with or without selection
// maps.  The arithmetic per pixel is that of the tile kernel (osbf_fwd2.cuh): running
// column sums a(y) = sum_{y-r..y} U in pass V, then the unrolled pass-H sweep with
// register rings forming the eight window sums of Eq. (6)-(13), the box kernels' means
// and Algorithm 2's selection; zeros beyond the padded frame come from the TMA fill (the
// appendix's boundary).  What differs is how the frame reaches shared memory:
//   * a persistent CTA owns segments: one plane, one strip of TW = 128 output columns
//     (+ r halo columns each side) and a run of 32-row chunks, walked top to bottom;
//   * the strip's rows arrive by TMA in boxes of 8 rows into a ring of NB boxes, each
//     slot with its own mbarrier; a box is issued as soon as the rows its slot held are
//     dead, a whole chunk before pass V needs it, so the copy latency is hidden;
//   * pass V keeps its running column sums in registers from chunk to chunk -- the
//     vertical halo is read once per segment instead of once per 32-row tile -- and works
//     in whole periods of r+1 rows (re-forming each sum from its register ring once per
//     period, as the tile kernel does), running up to r rows past the chunk;
//   * the column sums go to a ring of CH + 2r rows; pass H reads a(y), a(y+r) and U(y) of
//     its lane's row through per-lane ring offsets;
//   * frame-to-frame passes at r % 4 == 0 without maps write each lane's results from
//     registers, eight columns per 32-byte store (no staging buffer), which keeps the
//     shared memory at three CTAs per SM; the other launches stage rows per warp.
// The running sums re-form on the segment's row phase, not the tile's, so results can
// differ from the tile kernel's in the last bits (each is within the FP32 rule).
#pragma once

#include "osbf_fwd2.cuh"

namespace osbf {
namespace strip {

using v2::NT;
using v2::SW;
using v2::TW;
constexpr int CH = 32;   // rows per chunk: one pass-H row block (lane = row)
constexpr int BOXH = 8;  // rows per TMA box

struct StripParams {
    v2::Fwd2Params f;    // destination, maps, frame sizes, grid shift, error word
    int ys;              // frame row of the first output row (0 for frames, r for the output)
    int nchunks;         // chunks per strip
    int cps;             // chunks per segment
    int segs_per_strip;  // ceil(nchunks / cps)
    int strips_x;        // strips per plane
    int tx_off;          // index of the first strip (strip k starts at column (k + tx_off) * TW - tx_shift)
    int nsegs;           // planes * strips_x * segs_per_strip
};

struct StripLayout {
    int PU;        // float row pitch of both rings (PU % 8 == 4: conflict-free row-owner 16-byte access);
                   // the pass-H sweep of the last 32-column segment reads up to column 96 + 32 + 2r + 3
    int NB;        // TMA boxes in the U ring
    int MU, MA;    // rows of the U ring (NB boxes of 8 rows) and of the column-sum ring
    int box_bytes;
    int off_u, off_a, off_ms, off_xs, off_bar, bytes;
};

// Ring sizes.  Chunk c's pass H reads U rows [cCH + r, (c+1)CH + r) and column sums of rows
// [cCH + r, (c+1)CH + 2r); its pass V reads U rows up to (c+1)CH + 3r - 1 (whole periods).
// Row q of a segment (q = y - first row + r) sits in box q / 8.  When chunk c is done, boxes
// below ((c+1)CH + r) / 8 are dead; chunk c+2's pass V reaches box ((c+3)CH + 3r - 1) / 8, so
// NB = 9 + (3r - 1) / 8 - r / 8 slots let those loads start one chunk ahead.  Pass V of
// chunk c writes column sums up to row (c+1)CH + 3r - 1 while pass H(c) still needs row
// cCH + r: MA = CH + 2r.
constexpr int align128c(int b) { return (b + 127) & ~127; }

// constexpr: inside the kernels every ring size and offset is a compile-time constant
__host__ __device__ constexpr StripLayout make_strip_layout(int R, bool mstage, bool xstage) {
    StripLayout L{};
    L.PU = TW + 2 * R + 4;
    while (L.PU % 8 != 4) ++L.PU;
    L.NB = 9 + (3 * R - 1) / BOXH - R / BOXH;
    L.MU = L.NB * BOXH;
    L.MA = CH + 2 * R;
    L.box_bytes = L.PU * BOXH * 4;
    int off = 0;
    L.off_u = off;
    off = align128c(off + L.MU * L.PU * 4);
    L.off_a = off;
    off = align128c(off + L.MA * L.PU * 4);
    L.off_ms = off;
    if (mstage) off = align128c(off + (NT / 32) * 32 * v2::kMapPitch);
    L.off_xs = off;
    if (xstage) off = align128c(off + (NT / 32) * 32 * v2::kOutPitch * 4);
    L.off_bar = off;
    L.bytes = off + 8 * L.NB;
    return L;
}

// One period of pass V for this thread's column pair: rows q0 .. q0+R of the segment enter
// the running sums (U ring slots us.., column-sum ring slots as..).  The ring entry a row
// replaces is the row R+1 above it; the last row of the period re-forms the sum from the
// ring (the tile kernel's schedule, bounding FP32 drift).  GENERAL: a ring may wrap
// inside the period, or the period holds the segment's first rows (q < R: no full window
// yet, nothing stored).
template <int R, bool GENERAL>
__device__ __forceinline__ void period_v(const float *__restrict__ Ur, float *__restrict__ Ar, int pu, int us,
                                         int as, int q0, int MU, int MA, int c, float2 (&ring)[R + 1],
                                         float2 &acc) {
    constexpr int P = R + 1;
    float2 v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        int s = us + k;
        if (GENERAL && s >= MU) s -= MU;
        v[k] = *reinterpret_cast<const float2 *>(Ur + s * pu + c);
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (k == P - 1) {
            ring[k] = v[k];
            acc = ring[0];
#pragma unroll
            for (int i = 1; i < P; ++i) acc = v2::add2(acc, ring[i]);
        } else {
            acc = v2::add2(acc, v2::sub2(v[k], ring[k]));
            ring[k] = v[k];
        }
        if (!GENERAL || q0 + k >= R) {
            int s = as + k;
            if (GENERAL && s >= MA) s -= MA;
            *reinterpret_cast<float2 *>(Ar + s * pu + c) = acc;
        }
    }
}

// Kernel variants: MAPS (per-pass selection maps, staged per warp); V8 (r % 4 == 0, no
// maps, a destination whose strip columns start on 32 bytes: results leave from registers
// by 32-byte stores, three CTAs per SM); otherwise XSTAGE (results staged per warp and
// written a row at a time, any destination, two CTAs per SM).
template <int R, bool MAPS, bool V8>
__global__ void __launch_bounds__(NT, V8 ? 3 : 2)
    osbf_strip(const __grid_constant__ CUtensorMap src, const StripParams sp) {
    static_assert(!V8 || (R % 4 == 0 && !MAPS), "32-byte stores: r % 4 == 0, no maps");
    constexpr bool XSTAGE = !V8;
    constexpr int P = R + 1;
    extern __shared__ __align__(128) unsigned char smem_s[];
    const v2::Fwd2Params &p = sp.f;
    constexpr StripLayout L = make_strip_layout(R, MAPS, XSTAGE);
    float *Ur = reinterpret_cast<float *>(smem_s + L.off_u);
    float *Ar = reinterpret_cast<float *>(smem_s + L.off_a);
    const uint32_t bar0 = v2::smem_u32(smem_s + L.off_bar);
    const uint32_t ur0 = v2::smem_u32(Ur);
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int b = 0; b < L.NB; ++b) v2::mbar_init(bar0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        v2::fence_proxy_async();
    }
    __syncthreads();

    const int npairs = (TW + 2 * R + 1) / 2;  // pass V: one thread per column pair of the strip
    const bool vthread = tid < npairs;
    const int col = 2 * tid;
    unsigned gbox = 0;  // boxes this CTA issued before the current segment (ring slot and parity)
    for (int seg = blockIdx.x; seg < sp.nsegs; seg += gridDim.x) {
        const int per_plane = sp.strips_x * sp.segs_per_strip;
        const int plane = seg / per_plane;
        const int rem = seg - plane * per_plane;
        const int strip = rem / sp.segs_per_strip, sidx = rem - strip * sp.segs_per_strip;
        const int c0 = sidx * sp.cps;
        const int nch = sp.nchunks - c0 < sp.cps ? sp.nchunks - c0 : sp.cps;
        const int ys = sp.ys + c0 * CH;                       // frame row of the segment's first output
        const int tx0 = (strip + sp.tx_off) * TW - p.tx_shift;  // frame column of the strip's first output
        // row q of the segment is frame row ys - R + q; pass V reads whole periods of rows
        // until the last chunk's column sums exist: rows < P * ceil((nch*CH + 2R) / P)
        const int nbox = (P * ((nch * CH + 2 * R + P - 1) / P) - 1) / BOXH + 1;
        const unsigned gbase = gbox;
        gbox += nbox;
        int issued = 0, waited = 0;
        auto issue_upto = [&](int lim) {
            lim = lim < nbox ? lim : nbox;
            if (tid == 0 && issued < lim) {
                v2::fence_proxy_async();  // generic reads of the reused slots precede the copies
                for (int b = issued; b < lim; ++b) {
                    const int slot = (int)((gbase + b) % L.NB);
                    v2::tma_load_3d(ur0 + slot * L.box_bytes, &src, tx0 - R, ys - R + BOXH * b, plane,
                                    bar0 + 8 * slot, (uint32_t)L.box_bytes);
                }
            }
            if (issued < lim) issued = lim;
        };
        issue_upto(L.NB);  // every slot is free at a segment's start

        float2 ring[P], acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < P; ++k) ring[k] = make_float2(0.f, 0.f);
        int qv = 0;                                           // next row pass V consumes
        int us = (int)((gbase * BOXH) % L.MU), as = 0;        // its U-ring and column-sum-ring slots
        const int ubase = us;                                 // U-ring slot of row 0
        for (int ci = 0; ci < nch; ++ci) {
            // pass V: whole periods until the column sums of rows < ci*CH + CH + 2R exist
            const int target = ci * CH + CH + 2 * R;
            const int nper = target > qv ? (target - qv + P - 1) / P : 0;
            const int need = nper > 0 ? (qv + nper * P - 1) / BOXH + 1 : waited;
            bool timed_out = false;
            for (; waited < need; ++waited) {
                const unsigned gb = gbase + waited;
                if (!v2::mbar_wait_bounded(bar0 + 8 * (int)(gb % L.NB), (uint32_t)((gb / L.NB) & 1))) {
                    timed_out = true;
                    break;
                }
            }
            if (__syncthreads_or(timed_out)) {
                // report; thread 0 gives every copy still in flight one more bounded wait, so
                // shared memory outlives the copies that are merely late
                if (tid == 0) {
                    atomicOr(p.err, 1u);
                    for (int b = 0; b < issued; ++b) {
                        const unsigned gb = gbase + b;
                        v2::mbar_wait_bounded(bar0 + 8 * (int)(gb % L.NB), (uint32_t)((gb / L.NB) & 1));
                    }
                }
                return;
            }
            for (int k = 0; k < nper; ++k) {
                const bool general = qv < R || us + P > L.MU || as + P > L.MA;
                if (vthread) {
                    if (general)
                        period_v<R, true>(Ur, Ar, L.PU, us, as, qv, L.MU, L.MA, col, ring, acc);
                    else
                        period_v<R, false>(Ur, Ar, L.PU, us, as, qv, L.MU, L.MA, col, ring, acc);
                }
                qv += P;
                us += P;
                if (us >= L.MU) us -= L.MU;
                as += P;
                if (as >= L.MA) as -= L.MA;
            }
            __syncthreads();

            // pass H: warp w sweeps the strip's columns [32w, 32w + 32) of the chunk's 32 rows
            v2::Geom2 g;
            g.RHo = CH;
            g.RWo = TW;
            g.fy0 = ys + ci * CH;
            g.fx0 = tx0;
            g.FH = p.FH;
            g.FW = p.FW;
            g.iy0 = 0;
            g.iy1 = CH;
            g.ix0 = 0;
            g.ix1 = TW;
            g.oy = p.dst_is_output ? R : 0;
            g.ox = g.oy;
            g.ly = p.dst_is_output ? p.H : p.FH;
            g.lx = p.dst_is_output ? p.W : p.FW;
            g.MP = p.map_pitch;
            // this lane's row: q = ci*CH + R + lane; column sums a(q) and a(q + R), pixels U(q)
            const int q = ci * CH + R + lane;
            const int sa = (q % L.MA) * L.PU, sb = ((q + R) % L.MA) * L.PU;
            const int su = ((ubase + q) % L.MU) * L.PU;
            uint8_t *mplane = nullptr;
            if (MAPS && p.maps) mplane = p.maps + (long long)p.map_iter0 * p.map_iter_stride + (long long)plane * p.map_plane;
            float *gdst = reinterpret_cast<float *>(p.dst) + (long long)plane * p.dst_plane;
            v2::pass_h2<R, float, false, MAPS, true, false, false, XSTAGE, true, V8>(
                Ur, L.PU, 0, Ar, L.PU, nullptr, 0, gdst, p.dst_pitch, g, mplane, nullptr, nullptr, smem_s + L.off_ms,
                reinterpret_cast<float *>(smem_s + L.off_xs), sa, sb, su);
            __syncthreads();
            // rows below ((ci+1)CH + R) are dead: refill their slots
            issue_upto(((ci + 1) * CH + R) / BOXH + L.NB);
        }
        // every issued box has been waited for (each slot's phases are consumed in order);
        // this loop only runs if that ever stops holding
        for (; waited < issued; ++waited) {
            const unsigned gb = gbase + waited;
            if (!v2::mbar_wait_bounded(bar0 + 8 * (int)(gb % L.NB), (uint32_t)((gb / L.NB) & 1)) && tid == 0)
                atomicOr(p.err, 1u);
        }
        __syncthreads();
    }
}

template <int R, bool MAPS, bool V8>
cudaError_t launch_strip(const CUtensorMap &src, const StripParams &sp, int grid, cudaStream_t stream) {
    const StripLayout L = make_strip_layout(R, MAPS, !V8);
    auto kern = osbf_strip<R, MAPS, V8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, L.bytes, stream>>>(src, sp);
    return cudaGetLastError();
}

template <int R, bool MAPS, bool V8>
int occupancy_strip() {
    const StripLayout L = make_strip_layout(R, MAPS, !V8);
    auto kern = osbf_strip<R, MAPS, V8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT, L.bytes) != cudaSuccess) return 0;
    return n;
}

}  // namespace strip
}  // namespace osbf
