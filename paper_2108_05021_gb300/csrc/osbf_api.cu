// osbf_api.cu -- the C ABI of libosbf.so (see include/osbf.h): argument checks,
// workspace, the sequence of fused-group launches, host-buffer calls, tuning.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "osbf.h"
#include "osbf_internal.h"
#include "osbf_strip.cuh"

using namespace osbf;

struct osbf_ctx {
    int device = 0;
    int sms = 0;
    size_t smem_optin = 0;
    std::string err;
    void *frames[2] = {nullptr, nullptr};
    size_t frame_bytes[2] = {0, 0};
    void *dev_in = nullptr, *dev_out = nullptr;  // osbf_filter_host staging
    size_t dev_in_bytes = 0, dev_out_bytes = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;  // osbf_filter_host copy streams
    cudaEvent_t ev_start = nullptr, ev_in[4] = {}, ev_done[4] = {};
    void *ws[4] = {nullptr, nullptr, nullptr, nullptr};  // backward / checkpoint workspaces
    size_t ws_bytes[4] = {0, 0, 0, 0};
    int last_launches = 0;
    // (dtype, r, size class) -> the tuned forward: {fused depth, osbf_variant}
    std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
    void *batch_state = nullptr;                     // owned by the batched launcher
    unsigned int *err_word = nullptr;                // device: bit 0 = a bounded device wait gave up
    unsigned long long wait_ns = 0;                  // bound of the batched dependency wait (0 = default)
    int call_variant = 0;                            // forward kernel of the current call (osbf_variant)
    int call_fast = 0;                               // the current call runs the fast approximation
};

// implemented in osbf_bwd_api.cu / osbf_batched.cu
osbf_status osbf_backward_impl(osbf_ctx *ctx, const float *grad_out, float *grad_in, const uint8_t *maps, int P,
                               int H, int W, int r, int iters, cudaStream_t s);
void osbf_batched_free(osbf_ctx *ctx);

namespace {

osbf_status fail(osbf_ctx *ctx, osbf_status code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

#define OSBF_CK(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, OSBF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Runs a body with ctx->device current and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t elem_size(osbf_dtype dt) {
    switch (dt) {
    case OSBF_F32: return 4;
    case OSBF_F16: return 2;
    case OSBF_BF16: return 2;
    case OSBF_U8: return 1;
    }
    return 0;
}

Storage storage_of(osbf_dtype dt) {
    switch (dt) {
    case OSBF_F16: return Storage::F16;
    case OSBF_BF16: return Storage::BF16;
    case OSBF_U8: return Storage::U8;
    default: return Storage::F32;
    }
}

bool overlaps(const void *a, size_t an, const void *b, size_t bn) {
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + bn && pb < pa + an;
}

osbf_status ensure(osbf_ctx *ctx, void **slot, size_t *have, size_t need) {
    if (*have >= need) return OSBF_OK;
    if (*slot) cudaFree(*slot);
    *slot = nullptr;
    *have = 0;
    if (cudaMalloc(slot, need) != cudaSuccess) {
        cudaGetLastError();
        *slot = nullptr;
        return fail(ctx, OSBF_ENOMEM, "cudaMalloc of %zu bytes failed", need);
    }
    *have = need;
    return OSBF_OK;
}

// default fused depth before tuning: one pass per launch.  Measured on GB300 (4096^2 x 3,
// 30 passes, r in {1, 2, 4, 8, 16}), one pass per launch is the fastest for every radius:
// the kernel is bound by instruction issue, not by HBM, so fusing passes only adds the
// halo recomputation and the larger shared-memory footprint.
int default_depth(int r, osbf_dtype dt) {
    (void)r;
    (void)dt;
    return 1;
}

int size_class(long long pixels) {
    int c = 0;
    while (pixels > (1LL << 20) && c < 8) {
        pixels >>= 2;
        ++c;
    }
    return c;
}

}  // namespace

// ------------------------------------------------------------------------------------
// the forward driver (also used by the checkpointed forward and the backward's recompute)
// ------------------------------------------------------------------------------------
namespace {

size_t smem_v2(Storage st, int r, int D, bool direct = false) {
    switch (st) {
    case Storage::F16: return smem_fwd2_f16(r, D, direct);
    case Storage::BF16: return smem_fwd2_bf16(r, D, direct);
    default: return smem_fwd2_f32(r, D, direct);
    }
}

// largest fused depth <= D whose tile fits shared memory and the TMA box limits
int fit_depth(osbf_ctx *ctx, Storage st, int r, int D) {
    for (; D > 1; --D) {
        const int e = D * r;
        const int rw0 = v2::TW + 2 * round_up(e, st == Storage::F32 ? 4 : 8);
        if (smem_v2(st, r, D) <= ctx->smem_optin && rw0 + 16 <= 256 && v2::TH + 2 * e <= 256) break;
    }
    return D;
}

}  // namespace

namespace {

// One pass of the streaming strip kernel.  Strips use the tile kernel's column grid (the
// same shift); each strip's chunk rows are cut into segments so that the segments fill
// the grid in as few rounds as possible (a segment's start costs a pass-V warm-up of 2r
// rows and the first copy's latency, about one chunk).
cudaError_t launch_strip_group(const GroupLaunch &gl, int shift, cudaStream_t s, const char **what) {
    const int r = gl.r, P = gl.P, H = gl.H, W = gl.W;
    const int FH = H + 2 * r, FW = W + 2 * r;
    const bool last_out = gl.dst_is_output != 0;
    // 32-byte register stores where every strip's destination columns start on 32 bytes:
    // frames at r % 4 == 0 (no grid shift, pitch a multiple of 32 floats); the cropped
    // output at r % 8 == 0 with W % 8 == 0 and a 32-byte aligned base
    const bool v8 = !gl.maps && r % 4 == 0 &&
                    (!last_out || (r % 8 == 0 && W % 8 == 0 && ((uintptr_t)gl.dst & 31) == 0));
    strip::StripParams sp;
    std::memset(&sp, 0, sizeof sp);
    v2::Fwd2Params &p = sp.f;
    p.H = H;
    p.W = W;
    p.FH = FH;
    p.FW = FW;
    p.D = 1;
    p.maps = gl.maps;
    p.map_pitch = maps_pitch(FW);
    p.map_iter0 = gl.map_iter0;
    p.map_iter_stride = gl.map_iter_stride;
    p.map_plane = (long long)FH * p.map_pitch;
    p.err = gl.err;
    p.dst = gl.dst;
    p.dst_is_output = last_out ? 1 : 0;
    p.dst_pitch = last_out ? W : gl.dst_pitch;
    p.dst_plane = last_out ? (long long)H * W : (long long)FH * gl.dst_pitch;
    p.tx_shift = shift;
    // Every launch covers the whole frame with the same segments (the pass into the
    // cropped output clips its stores): the running sums re-form on the segment's row
    // phase, so with identical segments the map-writing, the plain and the output-writing
    // kernels compute every pixel identically.  The plan assumes three CTAs per SM (the
    // register-store kernels' occupancy) whatever the variant's, for the same reason.
    sp.ys = 0;
    sp.nchunks = (FH + strip::CH - 1) / strip::CH;
    sp.strips_x = (FW - 1 + shift) / v2::TW + 1;
    sp.tx_off = 0;
    int occ = occupancy_fwd_strip(r, gl.maps != nullptr, v8);
    if (occ < 1) occ = 1;
    const long long G = 3LL * gl.sms;
    const long long units = (long long)P * sp.strips_x;
    const double warm = 1.0 + 3.0 * r / strip::CH;  // chunk-equivalents per segment start
    double best = 1e300;
    for (int S = 1; S <= 64 && S <= sp.nchunks; ++S) {
        const int cps = (sp.nchunks + S - 1) / S;
        const int spp = (sp.nchunks + cps - 1) / cps;
        const long long nsegs = units * spp;
        const double cost = (double)((nsegs + G - 1) / G) * (cps + warm);
        if (cost < best - 1e-9) {
            best = cost;
            sp.cps = cps;
            sp.segs_per_strip = spp;
        }
    }
    const long long nsegs = units * sp.segs_per_strip;
    if (nsegs > 0x7fffffffLL) {
        *what = "too many segments";
        return cudaErrorInvalidValue;
    }
    sp.nsegs = (int)nsegs;
    CUtensorMap map;
    if (!encode_frame_map(&map, Storage::F32, gl.src, FW, FH, P, gl.src_pitch, strip_box_width(r), strip::BOXH)) {
        *what = "cuTensorMapEncodeTiled failed (source frame, strip boxes)";
        return cudaErrorInvalidValue;
    }
    const long long Gocc = (long long)occ * gl.sms;
    const int grid = (int)(Gocc < nsegs ? Gocc : nsegs);
    *what = "strip forward launch failed";
    return launch_fwd_strip(r, gl.maps != nullptr, v8, map, sp, grid, s);
}

}  // namespace

// One launch of the forward: `D` passes from the padded frame `src` into a frame or the
// caller's cropped output.  Every entry point that runs the float32 / 16-bit forward goes
// through here, so the choice of kernel variant, tile grid and summation order -- and
// with it the result, bit for bit -- is the same for all of them.
cudaError_t osbf::launch_group(const GroupLaunch &gl, cudaStream_t s, const char **what) {
    const Storage st = gl.st;
    const int r = gl.r, Dg = gl.D, P = gl.P, H = gl.H, W = gl.W;
    const int FH = H + 2 * r, FW = W + 2 * r;
    *what = "forward launch failed";
    // Direct: one pass written from registers (or staged rows) into the destination, a
    // frame or the cropped output; any r (the tile grid shifts so the halo stays exactly r
    // columns while the TMA box starts on 16 bytes).
    const bool last_out = gl.dst_is_output != 0;
    // the cropped output's rows hold aligned 4-vectors (16-bit kernels and tensor stores need them)
    const bool out_vec = W % 4 == 0 && r % 4 == 0 && ((uintptr_t)gl.dst % (st == Storage::F32 ? 16 : 8)) == 0;
    // float32 direct kernels without tensor stores stage their rows and write them one float
    // per lane, so they take any cropped output; their tile grid (shifted by (4 - r % 4) % 4)
    // and the fused-pass kernel's (halo rounded up to 4 columns) start every row segment on
    // the same frame column, so both give the same result bit for bit
    // (the fast approximation's direct kernel stores 4-vectors from registers: it needs out_vec)
    const bool out_ok = !last_out || (st == Storage::F32 && !gl.fast) || out_vec;
    // (the appendix tie order has single-pass kernels in float32 only)
    const bool direct = Dg == 1 && (gl.tie == 0 || st == Storage::F32) && out_ok;
    if (gl.fast && (!direct || st != Storage::F32 || gl.variant == 2)) {
        *what = "the fast approximation runs single float32 passes written from registers";
        return cudaErrorInvalidValue;
    }
    // float32 single passes at r % 4 == 0 of the paper tie order (no maps): results leave by
    // per-warp tensor stores of 32 x 32 segments -- into the next frame, or into the
    // cropped output when its rows hold whole 16-byte groups (W % 4 == 0, 16-byte aligned
    // base); frame-to-frame passes at r >= 8 take the early-load kernel instead (below)
    const bool tstore = direct && gl.tie == 0 && st == Storage::F32 && r % 4 == 0 && !gl.maps && (!last_out || out_vec);
    // The pass into the cropped output runs on the tile grid shifted by (r, r): tiles then
    // start at output rows 32k and columns 128k, so every tensor store starts at a
    // non-negative, 16-byte aligned output coordinate.  With maps the same grid, extended
    // by one tile row and column before the output, also covers the frame ring: the plain
    // and the map-writing passes share tile origins (and so their running sums' phases).
    const bool out_grid = last_out && direct && gl.tie == 0 && st == Storage::F32 && r % 4 == 0 && out_vec;
    const int shift = !direct ? 0 : st == Storage::F32 ? (4 - r % 4) % 4 : (8 - r % 8) % 8;
    // the streaming strip kernel: float32 single passes of the paper tie order at r <= 8; it
    // writes the cropped output through staged rows (one float per lane), so any W works
    const bool strip_ok = Dg == 1 && gl.tie == 0 && st == Storage::F32 && r <= OSBF_STRIP_MAX_R;
    // (opt-in: on GB300 it runs more instructions than the tile kernel -- its pass V works in
    // runtime loops of r+1-row periods over ring buffers -- and is slower at every radius)
    if (strip_ok && gl.variant == 2) return launch_strip_group(gl, (4 - r % 4) % 4, s, what);
    if (gl.variant == 2) {
        *what = "the streaming strip kernel does not cover this launch";
        return cudaErrorInvalidValue;
    }
    const v2::Layout2 L = st == Storage::F32   ? v2::make_layout2<float>(r, Dg, direct)
                          : st == Storage::F16 ? v2::make_layout2<__half>(r, Dg, direct)
                                               : v2::make_layout2<__nv_bfloat16>(r, Dg, direct);
    CUtensorMap map;
    if (gl.src_is_image) {
        // the padding first pass: the copy engine reads the unpadded image at frame
        // coordinates - r; the kernel replicates its border into the frame ring
        if (!tstore || gl.src_pitch != W) {
            *what = "a first pass from the unpadded image needs the tensor-store kernel";
            return cudaErrorInvalidValue;
        }
        if (!encode_frame_map(&map, st, gl.src, W, H, P, W, L.BX, L.RH0)) {
            *what = "cuTensorMapEncodeTiled failed (source image)";
            return cudaErrorInvalidValue;
        }
    } else if (!encode_frame_map(&map, st, gl.src, FW, FH, P, gl.src_pitch, L.BX, L.RH0)) {
        *what = "cuTensorMapEncodeTiled failed (source frame)";
        return cudaErrorInvalidValue;
    }
    v2::Fwd2Params p;
    std::memset(&p, 0, sizeof p);
    p.H = H;
    p.W = W;
    p.FH = FH;
    p.FW = FW;
    p.D = Dg;
    p.maps = gl.maps;
    p.map_pitch = maps_pitch(FW);
    p.map_iter0 = gl.map_iter0;
    p.map_iter_stride = gl.map_iter_stride;
    p.map_plane = (long long)FH * p.map_pitch;
    p.err = gl.err;
    p.dst = gl.dst;
    p.dst_is_output = last_out ? 1 : 0;
    p.dst_pitch = last_out ? W : gl.dst_pitch;
    p.dst_plane = last_out ? (long long)H * W : (long long)FH * gl.dst_pitch;
    p.src_off = gl.src_is_image ? r : 0;
    // tile k spans frame columns [k*TW - shift, (k+1)*TW - shift)
    int ty0 = 0, ty1 = (FH - 1) / v2::TH, tx0 = 0, tx1 = (FW - 1 + shift) / v2::TW;
    if (out_grid) {
        // tile k spans frame columns [k*TW + r, (k+1)*TW + r) (rows likewise)
        ty0 = gl.maps ? -1 : 0;
        tx0 = gl.maps ? -1 : 0;
        ty1 = gl.maps ? (FH - 1 - r) / v2::TH : (H - 1) / v2::TH;
        tx1 = gl.maps ? (FW - 1 - r) / v2::TW : (W - 1) / v2::TW;
    } else if (last_out && !gl.maps) {  // with maps, every frame pixel's selection is recorded
        ty0 = r / v2::TH;
        ty1 = (r + H - 1) / v2::TH;
        tx0 = (r + shift) / v2::TW;
        tx1 = (r + W - 1 + shift) / v2::TW;
    }
    p.ty_off = ty0;
    p.tx_off = tx0;
    p.tx_shift = out_grid ? -r : shift;
    p.ty_shift = out_grid ? -r : 0;
    p.tiles_x = tx1 - tx0 + 1;
    p.tiles_y = ty1 - ty0 + 1;
    CUtensorMap dmap;
    if (tstore && !(last_out ? encode_store_map(&dmap, p.dst, W, H, P, W)
                             : encode_store_map(&dmap, p.dst, FW, FH, P, p.dst_pitch))) {
        *what = "cuTensorMapEncodeTiled failed (store map)";
        return cudaErrorInvalidValue;
    }
    const long long ntiles = (long long)p.tiles_x * p.tiles_y * P;
    if (ntiles > 0x7fffffffLL) {
        *what = "too many tiles";
        return cudaErrorInvalidValue;
    }
    p.ntiles = (int)ntiles;
    // frame-to-frame passes of the tensor-store family at r >= 8 issue the next tile's load
    // before pass H and store from registers, 32 bytes at a time (same arithmetic, so the
    // same results bit for bit): the frame's row pitch and base lie on 32 bytes
    // (not for the fast approximation: with fewer instructions per pixel its passes are
    // bound by shared-memory throughput, which the 32-byte register stores load more than
    // the tensor stores do)
    const bool early = tstore && !last_out && !gl.src_is_image && !gl.fast && fwd2_early_radius(r) &&
                       gl.dst_pitch % 8 == 0 && ((uintptr_t)gl.dst & 31) == 0;
    int occ = early ? occupancy_fwd2_early(r, false) : tstore ? occupancy_fwd2_tstore(r, gl.fast != 0)
                     : gl.fast ? occupancy_fwd2_fast(r, gl.maps != nullptr)
                     : (st == Storage::F16    ? occupancy_fwd2_f16(r, gl.tie != 0, gl.maps != nullptr, direct, Dg)
                        : st == Storage::BF16 ? occupancy_fwd2_bf16(r, gl.tie != 0, gl.maps != nullptr, direct, Dg)
                                              : occupancy_fwd2_f32(r, gl.tie != 0, gl.maps != nullptr, direct, Dg));
    if (occ < 1) occ = 1;
    const long long g = (long long)occ * gl.sms;
    const int grid = (int)(g < ntiles ? g : ntiles);
    if (early) return launch_fwd2_early(r, false, map, p, grid, s);
    if (tstore) return launch_fwd2_tstore(r, gl.fast != 0, map, dmap, p, grid, s, gl.src_is_image != 0);
    if (gl.fast) return launch_fwd2_fast(r, gl.maps != nullptr, map, p, grid, s);
    switch (st) {
    case Storage::F16: return launch_fwd2_f16(r, gl.tie != 0, gl.maps != nullptr, direct, map, p, grid, s);
    case Storage::BF16: return launch_fwd2_bf16(r, gl.tie != 0, gl.maps != nullptr, direct, map, p, grid, s);
    default: return launch_fwd2_f32(r, gl.tie != 0, gl.maps != nullptr, direct, map, p, grid, s);
    }
}

// Runs `iters` passes.  `in` is the caller's image (in_is_frame = 0) or a padded frame
// of the storage type (in_is_frame = 1, row pitch in_pitch elements); `out` is the
// caller's cropped output (out_is_frame = 0) or a padded frame (pitch out_pitch).
osbf_status osbf_forward_run(osbf_ctx *ctx, const void *in, int in_is_frame, int in_pitch, void *out, int out_is_frame,
                             int out_pitch, int P, int H, int W, int r, int iters, osbf_dtype dtype, int depth,
                             int tie, uint8_t *maps, int maps_iter0, long long maps_iter_stride, cudaStream_t s) {
    // 8-bit input: the exact first pass writes a float32 frame; later passes run in float32
    const Storage st = dtype == OSBF_U8 ? Storage::F32 : storage_of(dtype);
    const int FH = H + 2 * r, FW = W + 2 * r;
    const size_t fes = st == Storage::F32 ? 4 : 2;  // frame element size
    const int align_el = (int)(128 / fes);
    const int FWp = (FW + align_el - 1) / align_el * align_el;
    const size_t frame_bytes = fes * (size_t)P * FH * FWp;
    const int MP = maps_pitch(FW);

    const bool fast = ctx->call_fast != 0;
    int D = fast ? 1 : depth > 0 ? depth : 0;
    int variant = fast ? (int)OSBF_VARIANT_TILE : ctx->call_variant;
    // the fast approximation writes the cropped output from registers only where its rows
    // hold aligned 4-vectors (r % 4 == 0, W % 4 == 0); otherwise its last pass writes a
    // frame and a crop follows
    const bool fast_crop = fast && !out_is_frame && !(W % 4 == 0 && r % 4 == 0 && ((uintptr_t)out & 15) == 0);
    if (D == 0) {
        // the tuned choice (osbf_autotune) applies when the caller fixed neither the depth
        // nor the kernel
        auto it = ctx->tuned.find(std::make_tuple((int)dtype, r, size_class((long long)P * H * W)));
        D = it != ctx->tuned.end() ? it->second.first : default_depth(r, dtype);
        if (variant == 0 && it != ctx->tuned.end()) variant = it->second.second;
    }
    if (D > OSBF_MAX_DEPTH) D = OSBF_MAX_DEPTH;
    D = fit_depth(ctx, st, r, D);
    // 16-bit single passes write the cropped output from registers only where its rows hold
    // aligned 4-vectors (r % 4 == 0, W % 4 == 0, base on 8 bytes); otherwise their last
    // pass writes a frame and a crop follows (the fused-pass kernel, the other way to
    // write the output, takes about three times as long for that pass; both start every
    // row segment on the same frame column, so the result is the same)
    const bool half_crop = st != Storage::F32 && !out_is_frame && D == 1 && tie == 0 &&
                           !(W % 4 == 0 && r % 4 == 0 && ((uintptr_t)out & 7) == 0);
    const bool crop_last = fast_crop || half_crop;
    if (smem_v2(st, r, 1) > ctx->smem_optin) return fail(ctx, OSBF_EUNSUPPORTED, "tile does not fit shared memory");

    // frame buffers: the padded input and the ping-pong targets
    void *fb[2] = {nullptr, nullptr};
    auto frame = [&](int k) -> void * {
        if (!fb[k]) {
            if (ensure(ctx, &ctx->frames[k], &ctx->frame_bytes[k], frame_bytes)) return nullptr;
            fb[k] = ctx->frames[k];
        }
        return fb[k];
    };

    const void *src = in;
    int src_pitch = in_pitch;
    int cur = -1;  // index of the frame buffer holding the current state (-1: the caller's)
    int passes = 0;
    // float32 tile passes at r % 4 == 0 (tensor stores, no maps): the first pass pads the
    // image itself (the copy engine reads the unpadded rows; the image's pitch W must hold
    // whole 16-byte groups), so no padding launch precedes it
    const bool pad_fused = !in_is_frame && dtype == OSBF_F32 && tie == 0 && !maps && D == 1 && r % 4 == 0 &&
                           W % 4 == 0 && ((uintptr_t)in & 15) == 0 && iters >= 2 && variant != OSBF_VARIANT_STRIP;
    if (!in_is_frame) {
        if (dtype == OSBF_U8) {
            // exact integer first pass (plain loads with replicate padding) into a float frame
            const bool direct = iters == 1 && !out_is_frame;
            FwdParams q;
            std::memset(&q, 0, sizeof q);
            q.src = in;
            q.src_is_input = 1;
            q.src_plane = (long long)H * W;
            q.src_pitch = W;
            q.H = H;
            q.W = W;
            q.FH = FH;
            q.FW = FW;
            q.D = 1;
            q.maps = maps;
            q.map_pitch = MP;
            q.map_iter0 = maps_iter0;
            q.map_iter_stride = maps_iter_stride;
            q.map_plane = (long long)FH * MP;
            void *dst = direct ? out : (iters == 1 ? out : frame(0));
            if (!dst) return OSBF_ENOMEM;
            q.dst = dst;
            q.dst_is_output = direct ? 1 : 0;
            q.dst_plane = direct ? (long long)H * W : (long long)FH * (iters == 1 ? out_pitch : FWp);
            q.dst_pitch = direct ? W : (iters == 1 ? out_pitch : FWp);
            int ty0 = 0, ty1 = (FH - 1) / kTH, tx0 = 0, tx1 = (FW - 1) / kTW;
            if (direct && !maps) {
                ty0 = r / kTH;
                ty1 = (r + H - 1) / kTH;
                tx0 = r / kTW;
                tx1 = (r + W - 1) / kTW;
            }
            q.ty_off = ty0;
            q.tx_off = tx0;
            for (int p0 = 0; p0 < P; p0 += 65535) {
                const int np = P - p0 < 65535 ? P - p0 : 65535;
                FwdParams qq = q;
                qq.src = (const uint8_t *)q.src + (size_t)p0 * q.src_plane;
                qq.dst = (float *)q.dst + (size_t)p0 * q.dst_plane;
                if (qq.maps) qq.maps = q.maps + (size_t)p0 * q.map_plane;
                cudaError_t e = launch_fwd_u8(r, tie != 0, qq, dim3(tx1 - tx0 + 1, ty1 - ty0 + 1, np), s);
                if (e != cudaSuccess) return fail(ctx, OSBF_ECUDA, "first-pass launch failed: %s", cudaGetErrorString(e));
                ctx->last_launches += 1;
            }
            passes = 1;
            if (iters == 1) return OSBF_OK;
            cur = 0;
            src = fb[0];
            src_pitch = FWp;
        } else if (pad_fused) {
            // the first pass reads the image itself and writes the padded frame's next state
            src = in;
            src_pitch = W;
        } else {
            void *f0 = frame(0);
            if (!f0) return OSBF_ENOMEM;
            cudaError_t e = launch_pad_replicate(st, in, f0, P, H, W, r, FH, FW, FWp, s);
            if (e != cudaSuccess) return fail(ctx, OSBF_ECUDA, "pad launch failed: %s", cudaGetErrorString(e));
            ctx->last_launches += 1;
            cur = 0;
            src = f0;
            src_pitch = FWp;
        }
    }

    while (passes < iters) {
        const int Dg = iters - passes < D ? iters - passes : D;
        const bool last = passes + Dg == iters;
        GroupLaunch gl;
        gl.st = st;
        gl.r = r;
        gl.D = Dg;
        gl.tie = tie;
        gl.src = src;
        gl.src_pitch = src_pitch;
        gl.P = P;
        gl.H = H;
        gl.W = W;
        gl.maps = maps;
        gl.map_iter0 = maps_iter0 + passes;
        gl.map_iter_stride = maps_iter_stride;
        gl.err = ctx->err_word;
        gl.sms = ctx->sms;
        gl.variant = variant;
        gl.src_is_image = pad_fused && passes == 0;
        gl.fast = fast ? 1 : 0;
        int nxt = -1;
        if (last && !out_is_frame && !crop_last) {
            gl.dst = out;
            gl.dst_is_output = 1;
        } else if (last && out_is_frame) {
            gl.dst = out;
            gl.dst_pitch = out_pitch;
        } else {
            nxt = cur == 0 ? 1 : 0;
            void *f = frame(nxt);
            if (!f) return OSBF_ENOMEM;
            gl.dst = f;
            gl.dst_pitch = FWp;
        }
        const char *what = nullptr;
        cudaError_t e = launch_group(gl, s, &what);
        if (e != cudaSuccess) return fail(ctx, OSBF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
        ctx->last_launches += 1;
        passes += Dg;
        if (nxt >= 0) {
            cur = nxt;
            src = fb[nxt];
            src_pitch = FWp;
        }
    }
    if (crop_last) {
        cudaError_t e = st == Storage::F32 ? launch_crop_f32((const float *)fb[cur], (float *)out, P, H, W, r, FWp, s)
                                           : launch_crop_16(fb[cur], out, P, H, W, r, FWp, s);
        if (e != cudaSuccess) return fail(ctx, OSBF_ECUDA, "crop launch failed: %s", cudaGetErrorString(e));
        ctx->last_launches += 1;
    }
    return OSBF_OK;
}

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" {

const char *osbf_version(void) { return "osbf-gb300 0.1 (sm_103a)"; }

osbf_status osbf_create(osbf_ctx **out, int device) {
    if (!out) return OSBF_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return device < 0 ? OSBF_EINVAL : OSBF_ECUDA;
    }
    osbf_ctx *ctx = new (std::nothrow) osbf_ctx();
    if (!ctx) return OSBF_ENOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    ctx->sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->smem_optin = (size_t)v;
    if (cudaMalloc(&ctx->err_word, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(ctx->err_word, 0, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return OSBF_ENOMEM;
    }
    *out = ctx;
    return OSBF_OK;
}

void osbf_destroy(osbf_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (void *p : ctx->frames)
        if (p) cudaFree(p);
    for (void *p : ctx->ws)
        if (p) cudaFree(p);
    if (ctx->dev_in) cudaFree(ctx->dev_in);
    if (ctx->dev_out) cudaFree(ctx->dev_out);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    for (int k = 0; k < 4; ++k) {
        if (ctx->ev_in[k]) cudaEventDestroy(ctx->ev_in[k]);
        if (ctx->ev_done[k]) cudaEventDestroy(ctx->ev_done[k]);
    }
    if (ctx->err_word) cudaFree(ctx->err_word);
    osbf_batched_free(ctx);
    delete ctx;
}

const char *osbf_last_error(const osbf_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int osbf_last_launch_count(const osbf_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

osbf_status osbf_set_wait_timeout(osbf_ctx *ctx, unsigned long long ns) {
    if (!ctx) return OSBF_EINVAL;
    ctx->wait_ns = ns;
    return OSBF_OK;
}

osbf_status osbf_check(osbf_ctx *ctx) {
    if (!ctx) return OSBF_EINVAL;
    DeviceGuard g(ctx->device);
    OSBF_CK(cudaDeviceSynchronize());
    unsigned int w = 0;
    OSBF_CK(cudaMemcpy(&w, ctx->err_word, sizeof w, cudaMemcpyDeviceToHost));
    if (w) {
        OSBF_CK(cudaMemset(ctx->err_word, 0, sizeof w));
        return fail(ctx, OSBF_ETIMEOUT, "a bounded device-side wait gave up (error word 0x%x)", w);
    }
    return OSBF_OK;
}

osbf_status osbf_filter_ex(osbf_ctx *ctx, const void *in, void *out, int N, int C, int H, int W, int r, int iters,
                           osbf_dtype dtype, const osbf_options *opts, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    ctx->err.clear();
    ctx->last_launches = 0;
    if (!in || !out) return fail(ctx, OSBF_EINVAL, "null image pointer");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0) return fail(ctx, OSBF_EINVAL, "N, C, H and W must be positive");
    if (r < 0 || iters < 0) return fail(ctx, OSBF_EINVAL, "r and iters must be >= 0");
    if (dtype < OSBF_F32 || dtype > OSBF_U8) return fail(ctx, OSBF_EINVAL, "unknown dtype %d", (int)dtype);
    osbf_options o;
    std::memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.depth < 0 || o.depth > OSBF_MAX_DEPTH) return fail(ctx, OSBF_EINVAL, "depth must be in 0..%d", OSBF_MAX_DEPTH);
    if (o.tie != OSBF_TIE_PAPER && o.tie != OSBF_TIE_APPENDIX) return fail(ctx, OSBF_EINVAL, "unknown tie order");
    for (int v : o.reserved)
        if (v) return fail(ctx, OSBF_EINVAL, "reserved option fields must be zero");
    if (o.variant < OSBF_VARIANT_AUTO || o.variant > OSBF_VARIANT_STRIP)
        return fail(ctx, OSBF_EINVAL, "unknown forward variant %d", o.variant);
    if (o.variant == OSBF_VARIANT_STRIP && (r > OSBF_STRIP_MAX_R || o.tie != OSBF_TIE_PAPER || dtype == OSBF_F16 ||
                                            dtype == OSBF_BF16 || o.depth > 1))
        return fail(ctx, OSBF_EUNSUPPORTED, "the strip kernel runs float32 single passes, paper tie order, r <= %d",
                    OSBF_STRIP_MAX_R);
    if (r > OSBF_MAX_RADIUS) return fail(ctx, OSBF_EUNSUPPORTED, "r = %d exceeds OSBF_MAX_RADIUS = %d", r, OSBF_MAX_RADIUS);
    if (o.maps && (dtype == OSBF_F16 || dtype == OSBF_BF16) && o.tie != OSBF_TIE_PAPER)
        return fail(ctx, OSBF_EUNSUPPORTED, "16-bit storage keeps selection maps with the paper tie order only");
    const long long P = (long long)N * C;
    if (P * H * (long long)W > (1LL << 40)) return fail(ctx, OSBF_EUNSUPPORTED, "image too large");
    const size_t in_bytes = elem_size(dtype) * (size_t)P * H * W;
    const size_t out_bytes = (dtype == OSBF_U8 ? 4 : elem_size(dtype)) * (size_t)P * H * W;
    if (overlaps(in, in_bytes, out, out_bytes)) return fail(ctx, OSBF_EINVAL, "in and out overlap");
    const int FH = H + 2 * r, FW = W + 2 * r;
    const long long map_stride = P * FH * maps_pitch(FW);
    if (o.maps && ((uintptr_t)o.maps & 15)) return fail(ctx, OSBF_EINVAL, "maps must be 16-byte aligned");
    if (o.maps && iters > 0 && (overlaps(o.maps, (size_t)map_stride * iters, in, in_bytes) ||
                                overlaps(o.maps, (size_t)map_stride * iters, out, out_bytes)))
        return fail(ctx, OSBF_EINVAL, "maps overlap an image");

    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0 || iters == 0) {
        // every window is the centre pixel (r = 0) or no pass runs: the input itself
        if (dtype == OSBF_U8) {
            OSBF_CK(launch_u8_to_f32((const uint8_t *)in, (float *)out, P * H * W, s));
        } else {
            OSBF_CK(cudaMemcpyAsync(out, in, in_bytes, cudaMemcpyDeviceToDevice, s));
        }
        ctx->last_launches = 1;
        if (o.maps && iters > 0) {
            // all |d_i| are 0: the first window of the tie order is selected everywhere
            const uint8_t first = o.tie == OSBF_TIE_APPENDIX ? 6 : 1;
            OSBF_CK(launch_fill_u8(o.maps, first, map_stride * iters, s));
            ctx->last_launches += 1;
        }
        return OSBF_OK;
    }
    ctx->call_variant = o.variant;
    const osbf_status st = osbf_forward_run(ctx, in, 0, 0, out, 0, 0, (int)P, H, W, r, iters, dtype, o.depth, o.tie,
                                            o.maps, 0, map_stride, s);
    ctx->call_variant = 0;
    return st;
}

osbf_status osbf_filter(osbf_ctx *ctx, const void *in, void *out, int N, int C, int H, int W, int r, int iters,
                        osbf_dtype dtype, void *stream) {
    return osbf_filter_ex(ctx, in, out, N, C, H, W, r, iters, dtype, nullptr, stream);
}

osbf_status osbf_filter_host(osbf_ctx *ctx, const void *in, void *out, int N, int C, int H, int W, int r, int iters,
                             osbf_dtype dtype, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    ctx->err.clear();
    if (!in || !out) return fail(ctx, OSBF_EINVAL, "null image pointer");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0) return fail(ctx, OSBF_EINVAL, "N, C, H and W must be positive");
    if (dtype < OSBF_F32 || dtype > OSBF_U8) return fail(ctx, OSBF_EINVAL, "unknown dtype %d", (int)dtype);
    const long long P = (long long)N * C;
    const size_t in_bytes = elem_size(dtype) * (size_t)P * H * W;
    const size_t out_bytes = (dtype == OSBF_U8 ? 4 : elem_size(dtype)) * (size_t)P * H * W;
    DeviceGuard g(ctx->device);
    osbf_status e = ensure(ctx, &ctx->dev_in, &ctx->dev_in_bytes, in_bytes);
    if (e) return e;
    e = ensure(ctx, &ctx->dev_out, &ctx->dev_out_bytes, out_bytes);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)stream;
    // Planes are independent: up to four plane chunks, each copied in on one stream,
    // filtered on the caller's stream once its copy has landed, and copied out on a third
    // stream once filtered -- the copies of one chunk overlap the filtering of another.
    if (!ctx->copy_in) {
        OSBF_CK(cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
        OSBF_CK(cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
        OSBF_CK(cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
        for (int k = 0; k < 4; ++k) {
            OSBF_CK(cudaEventCreateWithFlags(&ctx->ev_in[k], cudaEventDisableTiming));
            OSBF_CK(cudaEventCreateWithFlags(&ctx->ev_done[k], cudaEventDisableTiming));
        }
    }
    const int K = (int)std::min<long long>(P, 4);
    const size_t pin = in_bytes / (size_t)P, pout = out_bytes / (size_t)P;  // bytes per plane
    // the staging buffers are free once the caller's stream has finished earlier work
    OSBF_CK(cudaEventRecord(ctx->ev_start, s));
    OSBF_CK(cudaStreamWaitEvent(ctx->copy_in, ctx->ev_start, 0));
    OSBF_CK(cudaStreamWaitEvent(ctx->copy_out, ctx->ev_start, 0));
    long long p0[5];
    for (int c = 0; c <= K; ++c) p0[c] = P * c / K;
    for (int c = 0; c < K; ++c) {
        OSBF_CK(cudaMemcpyAsync((char *)ctx->dev_in + p0[c] * pin, (const char *)in + p0[c] * pin,
                                (size_t)(p0[c + 1] - p0[c]) * pin, cudaMemcpyHostToDevice, ctx->copy_in));
        OSBF_CK(cudaEventRecord(ctx->ev_in[c], ctx->copy_in));
    }
    int launches = 0;
    for (int c = 0; c < K; ++c) {
        OSBF_CK(cudaStreamWaitEvent(s, ctx->ev_in[c], 0));
        e = osbf_filter_ex(ctx, (const char *)ctx->dev_in + p0[c] * pin, (char *)ctx->dev_out + p0[c] * pout,
                           (int)(p0[c + 1] - p0[c]), 1, H, W, r, iters, dtype, nullptr, stream);
        if (e) {
            cudaStreamSynchronize(ctx->copy_in);
            cudaStreamSynchronize(ctx->copy_out);
            return e;
        }
        launches += ctx->last_launches;
        OSBF_CK(cudaEventRecord(ctx->ev_done[c], s));
        OSBF_CK(cudaStreamWaitEvent(ctx->copy_out, ctx->ev_done[c], 0));
        OSBF_CK(cudaMemcpyAsync((char *)out + p0[c] * pout, (const char *)ctx->dev_out + p0[c] * pout,
                                (size_t)(p0[c + 1] - p0[c]) * pout, cudaMemcpyDeviceToHost, ctx->copy_out));
    }
    ctx->last_launches = launches;
    OSBF_CK(cudaStreamSynchronize(ctx->copy_out));
    OSBF_CK(cudaStreamSynchronize(s));
    unsigned int w = 0;
    OSBF_CK(cudaMemcpy(&w, ctx->err_word, sizeof w, cudaMemcpyDeviceToHost));
    if (w) {
        cudaMemset(ctx->err_word, 0, sizeof w);
        return fail(ctx, OSBF_ETIMEOUT, "a bounded device-side wait gave up");
    }
    return OSBF_OK;
}

osbf_status osbf_autotune(osbf_ctx *ctx, osbf_dtype dtype, int planes, int H, int W, int r, int iters) {
    if (!ctx) return OSBF_EINVAL;
    ctx->err.clear();
    if (planes <= 0 || H <= 0 || W <= 0 || r < 1 || iters < 1) return fail(ctx, OSBF_EINVAL, "bad tuning problem");
    if (r > OSBF_MAX_RADIUS) return fail(ctx, OSBF_EUNSUPPORTED, "r exceeds OSBF_MAX_RADIUS");
    if (dtype < OSBF_F32 || dtype > OSBF_U8) return fail(ctx, OSBF_EINVAL, "unknown dtype");
    DeviceGuard g(ctx->device);
    const size_t in_bytes = elem_size(dtype) * (size_t)planes * H * W;
    const size_t out_bytes = (dtype == OSBF_U8 ? 4 : elem_size(dtype)) * (size_t)planes * H * W;
    void *din = nullptr, *dout = nullptr;
    if (cudaMalloc(&din, in_bytes) != cudaSuccess || cudaMalloc(&dout, out_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (din) cudaFree(din);
        return fail(ctx, OSBF_ENOMEM, "tuning buffers");
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Storage st = storage_of(dtype);
    osbf_status status = OSBF_OK;
    if (launch_tuning_image(st, din, planes, H, W, s) != cudaSuccess)
        status = fail(ctx, OSBF_ECUDA, "tuning image fill failed");
    // candidates: the tile kernel at every fused depth that fits (a larger requested depth
    // is clamped to the largest that fits, so stop at the first clamped one), and the
    // streaming strip kernel for float32 single passes
    std::vector<std::pair<int, int>> cand;  // {depth, variant}
    const Storage fst = dtype == OSBF_U8 ? Storage::F32 : st;
    for (int D = 1; D <= OSBF_MAX_DEPTH && D <= iters; ++D) {
        if (fit_depth(ctx, fst, r, D) != D) break;
        cand.push_back({D, OSBF_VARIANT_TILE});
    }
    if ((dtype == OSBF_F32 || dtype == OSBF_U8) && r <= OSBF_STRIP_MAX_R) cand.push_back({1, OSBF_VARIANT_STRIP});
    std::pair<int, int> best = {1, OSBF_VARIANT_TILE};
    float best_ms = 1e30f;
    for (size_t c = 0; c < cand.size() && status == OSBF_OK; ++c) {
        osbf_options o;
        std::memset(&o, 0, sizeof o);
        o.depth = cand[c].first;
        o.variant = cand[c].second;
        status = osbf_filter_ex(ctx, din, dout, planes, 1, H, W, r, iters, dtype, &o, s);  // warm-up
        if (status) break;
        cudaEventRecord(e0, s);
        const int reps = 3;
        for (int k = 0; k < reps && !status; ++k)
            status = osbf_filter_ex(ctx, din, dout, planes, 1, H, W, r, iters, dtype, &o, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (status) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(din);
    cudaFree(dout);
    if (status) return status;
    ctx->tuned[std::make_tuple((int)dtype, r, size_class((long long)planes * H * W))] = best;
    return OSBF_OK;
}

osbf_status osbf_set_tuned(osbf_ctx *ctx, osbf_dtype dtype, int planes, int H, int W, int r, int depth, int variant) {
    if (!ctx) return OSBF_EINVAL;
    ctx->err.clear();
    if (planes <= 0 || H <= 0 || W <= 0 || r < 1 || r > OSBF_MAX_RADIUS || dtype < OSBF_F32 || dtype > OSBF_U8)
        return fail(ctx, OSBF_EINVAL, "bad tuning key");
    if (depth < 1 || depth > OSBF_MAX_DEPTH || variant < OSBF_VARIANT_TILE || variant > OSBF_VARIANT_STRIP)
        return fail(ctx, OSBF_EINVAL, "bad tuned choice");
    if (variant == OSBF_VARIANT_STRIP &&
        (depth != 1 || r > OSBF_STRIP_MAX_R || dtype == OSBF_F16 || dtype == OSBF_BF16))
        return fail(ctx, OSBF_EUNSUPPORTED, "the strip kernel runs float32 single passes at r <= %d", OSBF_STRIP_MAX_R);
    ctx->tuned[std::make_tuple((int)dtype, r, size_class((long long)planes * H * W))] = {depth, variant};
    return OSBF_OK;
}

osbf_status osbf_tuned(osbf_ctx *ctx, osbf_dtype dtype, int planes, int H, int W, int r, int *depth, int *variant) {
    if (!ctx || !depth || !variant) return OSBF_EINVAL;
    auto it = ctx->tuned.find(std::make_tuple((int)dtype, r, size_class((long long)planes * H * W)));
    if (it == ctx->tuned.end()) {
        *depth = 0;
        *variant = OSBF_VARIANT_AUTO;
        return OSBF_OK;
    }
    *depth = it->second.first;
    *variant = it->second.second;
    return OSBF_OK;
}

osbf_status osbf_filter_fast(osbf_ctx *ctx, const float *in, float *out, int N, int C, int H, int W, int r, int iters,
                             uint8_t *maps, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    ctx->err.clear();
    ctx->last_launches = 0;
    if (!in || !out) return fail(ctx, OSBF_EINVAL, "null image pointer");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0) return fail(ctx, OSBF_EINVAL, "N, C, H and W must be positive");
    if (r < 0 || iters < 0) return fail(ctx, OSBF_EINVAL, "r and iters must be >= 0");
    if (r > OSBF_MAX_RADIUS) return fail(ctx, OSBF_EUNSUPPORTED, "r = %d exceeds OSBF_MAX_RADIUS = %d", r, OSBF_MAX_RADIUS);
    if (maps && ((uintptr_t)maps & 15)) return fail(ctx, OSBF_EINVAL, "maps must be 16-byte aligned");
    const long long P = (long long)N * C;
    if (P * H * (long long)W > (1LL << 40)) return fail(ctx, OSBF_EUNSUPPORTED, "image too large");
    const size_t bytes = 4 * (size_t)P * H * W;
    if (overlaps(in, bytes, out, bytes)) return fail(ctx, OSBF_EINVAL, "in and out overlap");
    const int FH = H + 2 * r, FW = W + 2 * r, FWp = (FW + 31) / 32 * 32, MP = maps_pitch(FW);
    const long long map_stride = P * FH * MP;
    if (maps && iters > 0 && (overlaps(maps, (size_t)map_stride * iters, in, bytes) ||
                              overlaps(maps, (size_t)map_stride * iters, out, bytes)))
        return fail(ctx, OSBF_EINVAL, "maps overlap an image");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0 || iters == 0) {
        OSBF_CK(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s));
        ctx->last_launches = 1;
        if (maps && iters > 0) {  // every candidate equals the pixel: N1, first in the paper order
            OSBF_CK(launch_fill_u8(maps, 1, map_stride * iters, s));
            ctx->last_launches += 1;
        }
        return OSBF_OK;
    }
    // the float32 forward's launch plan (padding first pass, output-aligned last pass,
    // shared tile origins for the plain and the map-writing calls) with the fast kernels
    ctx->call_fast = 1;
    const osbf_status st = osbf_forward_run(ctx, in, 0, 0, out, 0, 0, (int)P, H, W, r, iters, OSBF_F32, 1, 0, maps, 0,
                                            map_stride, s);
    ctx->call_fast = 0;
    return st;
}

osbf_status osbf_filter_backward(osbf_ctx *ctx, const float *grad_out, float *grad_in, const uint8_t *maps, int N,
                                 int C, int H, int W, int r, int iters, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    ctx->err.clear();
    ctx->last_launches = 0;
    if (!grad_out || !grad_in || (!maps && iters > 0 && r > 0)) return fail(ctx, OSBF_EINVAL, "null pointer");
    if (maps && ((uintptr_t)maps & 15)) return fail(ctx, OSBF_EINVAL, "maps must be 16-byte aligned");
    if (N <= 0 || C <= 0 || H <= 0 || W <= 0) return fail(ctx, OSBF_EINVAL, "N, C, H and W must be positive");
    if (r < 0 || iters < 0) return fail(ctx, OSBF_EINVAL, "r and iters must be >= 0");
    if (r > OSBF_MAX_RADIUS) return fail(ctx, OSBF_EUNSUPPORTED, "r exceeds OSBF_MAX_RADIUS");
    const long long P = (long long)N * C;
    const size_t bytes = 4 * (size_t)P * H * W;
    if (overlaps(grad_out, bytes, grad_in, bytes)) return fail(ctx, OSBF_EINVAL, "grad_out and grad_in overlap");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0 || iters == 0) {
        OSBF_CK(cudaMemcpyAsync(grad_in, grad_out, bytes, cudaMemcpyDeviceToDevice, s));
        ctx->last_launches = 1;
        return OSBF_OK;
    }
    return osbf_backward_impl(ctx, grad_out, grad_in, maps, (int)P, H, W, r, iters, s);
}

}  // extern "C"

// accessors for the other translation units
unsigned int *osbf_ctx_err_word(osbf_ctx *ctx) { return ctx->err_word; }
unsigned long long osbf_ctx_wait_ns(const osbf_ctx *ctx) { return ctx->wait_ns; }
int osbf_ctx_tuned_depth(osbf_ctx *ctx, osbf_dtype dt, int r, long long pixels) {
    auto it = ctx->tuned.find(std::make_tuple((int)dt, r, size_class(pixels)));
    return it != ctx->tuned.end() ? it->second.first : default_depth(r, dt);
}
// a tuned float32 choice other than the tile kernel at depth 1 (the batched launch's own)
bool osbf_ctx_tuned_elsewhere(osbf_ctx *ctx, int r, long long pixels) {
    auto it = ctx->tuned.find(std::make_tuple((int)OSBF_F32, r, size_class(pixels)));
    return it != ctx->tuned.end() && (it->second.first != 1 || it->second.second == OSBF_VARIANT_STRIP);
}
void *osbf_ctx_workspace(osbf_ctx *ctx, int slot, size_t bytes, osbf_status *st) {
    *st = ensure(ctx, &ctx->ws[slot], &ctx->ws_bytes[slot], bytes);
    return *st == OSBF_OK ? ctx->ws[slot] : nullptr;
}
osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg) { return fail(ctx, code, "%s", msg); }
void osbf_ctx_count_launches(osbf_ctx *ctx, int n) { ctx->last_launches += n; }
void osbf_ctx_reset_launches(osbf_ctx *ctx) {
    ctx->last_launches = 0;
    ctx->err.clear();
}
int osbf_ctx_sms(const osbf_ctx *ctx) { return ctx->sms; }
int osbf_ctx_device(const osbf_ctx *ctx) { return ctx->device; }
void **osbf_ctx_batch_state(osbf_ctx *ctx) { return &ctx->batch_state; }
