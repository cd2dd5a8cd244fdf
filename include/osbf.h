/*
 * osbf.h -- C ABI of the GB300 One-Sided Box Filter library (libosbf.so).
 *
 * The filter is the One-Sided Box Filter of Gong, "One-Sided Box Filter for Edge
 * Preserving Image Smoothing" (arxiv 2108.05021):
 *   - Eq. (1): U = Phi(I(N(x, y))), here Phi = mean over one of eight windows;
 *   - Eq. (6)-(13): the eight one-sided windows N1..N8 of radius r around (x, y)
 *     (N1-N4 quadrants of (r+1)^2 pixels, N5-N8 half windows of (r+1)(2r+1));
 *   - Sec. "One-sided Kernels for Box Filter": the box kernels k1..k8 (a window
 *     mean normalised by the full window size);
 *   - Algorithm 2: d_i = k_i (x) U - U, m = argmin_i |d_i|, U <- U + d_m, repeated;
 *   - the appendix listing: the image is replicate-padded by r once, every pass
 *     runs on the padded frame with zeros beyond it (the frame's ring evolves
 *     too), and the result is the frame cropped back to H x W.
 * Coordinates: x = column (the W axis), y = row (the H axis, increasing down).
 * `iters` passes are run (the appendix's loop count).  Ties in |d_i| go to the
 * first window in the tie order (OSBF_TIE_PAPER: N1..N8; OSBF_TIE_APPENDIX:
 * the appendix's difference planes N6, N5, N7, N8, N2, N1, N3, N4).
 *
 * Conventions for every entry point:
 *   - Images are N x C x H x W, contiguous, row-major (NCHW).  Every channel is a
 *     separate plane, filtered independently (the appendix loops over channels).
 *   - Unless a function says otherwise, image, gradient and map pointers are
 *     DEVICE pointers on the context's device, owned by the caller, and must not
 *     alias each other.
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = the legacy default
 *     stream) and is asynchronous unless stated otherwise.
 *   - Errors come back as osbf_status codes; no exception crosses the ABI.  The
 *     text of the last error of a context is returned by osbf_last_error().
 *   - A context is not thread-safe: use one context per host thread.  Its calls share
 *     its workspaces: calls on different streams must not overlap on the GPU (order
 *     the streams with events, or use one context per stream).
 *   - Radii 0..OSBF_MAX_RADIUS are supported; larger r gives OSBF_EUNSUPPORTED.
 *     r = 0 or iters = 0 returns the input unchanged (converted to the output
 *     type for 8-bit input).
 */
#ifndef OSBF_H
#define OSBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OSBF_MAX_RADIUS 16
#define OSBF_MAX_DEPTH 8

typedef enum {
    OSBF_OK = 0,
    OSBF_EINVAL = 1,       /* a bad argument (null pointer, non-positive size, aliasing, ...) */
    OSBF_ENOMEM = 2,       /* a workspace allocation failed */
    OSBF_ECUDA = 3,        /* a CUDA runtime or driver call failed */
    OSBF_EUNSUPPORTED = 4, /* valid but not supported (r > OSBF_MAX_RADIUS, dtype, ...) */
    OSBF_ETIMEOUT = 5      /* a bounded device-side wait gave up (outputs of that call undefined) */
} osbf_status;

typedef enum {
    OSBF_F32 = 0,  /* float32 storage and arithmetic */
    OSBF_F16 = 1,  /* float16 storage; sums and scores in float32, rounded to f16 after every pass */
    OSBF_BF16 = 2, /* bfloat16 storage; as OSBF_F16 */
    OSBF_U8 = 3    /* uint8 input, float32 output; first pass exact in integers (see below) */
} osbf_dtype;

typedef enum { OSBF_TIE_PAPER = 0, OSBF_TIE_APPENDIX = 1 } osbf_tie;

typedef struct osbf_ctx osbf_ctx;

/* Per-call options of osbf_filter_ex().  Zero-initialise, then set fields. */
typedef struct {
    int depth;       /* passes fused per launch (temporal blocking), 1..OSBF_MAX_DEPTH;
                        0 = the tuned choice for (dtype, r, size) */
    int tie;         /* osbf_tie */
    uint8_t *maps;   /* optional device buffer, iters x N*C x (H+2r) rows of
                        osbf_maps_pitch(W, r) bytes, 16-byte aligned: the selected window
                        index (1..8 = N1..N8) of every frame pixel and pass in the first
                        W+2r bytes of each row (the rest of the row is unspecified) */
    int variant;     /* forward kernel (osbf_variant); 0 = the library's choice */
    int reserved[3]; /* must be zero */
} osbf_options;

/* Forward kernels of the float32 single-pass launches (paper tie order).  Both compute the
 * same filter; they differ in the last bits of the running sums, so a call runs all its
 * passes with one of them.  OSBF_VARIANT_STRIP covers r <= 8 (OSBF_EUNSUPPORTED above). */
typedef enum {
    OSBF_VARIANT_AUTO = 0,  /* the tuned choice (osbf_autotune), else the tile kernel */
    OSBF_VARIANT_TILE = 1,  /* 32 x 128 tiles, each loaded with its halo by one tensor copy */
    OSBF_VARIANT_STRIP = 2  /* column strips streamed top to bottom in 32-row chunks, copies a chunk ahead */
} osbf_variant;

/* Create a context on CUDA device `device`.  *out receives it.  The context owns
 * workspaces (two padded frames per shape class, grown on demand), the tuned
 * choices and the batched launch's graphs; osbf_destroy() frees them. */
osbf_status osbf_create(osbf_ctx **out, int device);

/* Destroy a context (synchronises the device first).  NULL is ignored. */
void osbf_destroy(osbf_ctx *ctx);

/* Text of the last error recorded in `ctx` ("" if none).  Valid until the next call. */
const char *osbf_last_error(const osbf_ctx *ctx);

/*
 * Forward filter (Algorithm 2 with the appendix's boundary; see the file comment).
 *   in    N x C x H x W, element type per `dtype` (uint8 for OSBF_U8).
 *   out   N x C x H x W, same element type as `in`, except float32 for OSBF_U8
 *         (the appendix works in single precision).
 * OSBF_U8: the first pass is exact: integer window sums S_i, the selection
 * compares |S_i - n_i U| n_j with |S_j - n_j U| n_i in int64, and the new value is
 * the correctly rounded float32 of S_m / n_m; later passes run in float32.
 * Returns OSBF_EINVAL for null pointers, N, C, H or W <= 0, r or iters < 0, or
 * in == out; OSBF_EUNSUPPORTED for r > OSBF_MAX_RADIUS.
 */
osbf_status osbf_filter(osbf_ctx *ctx, const void *in, void *out, int N, int C, int H, int W, int r, int iters,
                        osbf_dtype dtype, void *stream);

/* osbf_filter() with options (fused depth, tie order, selection maps).  opts may be NULL. */
osbf_status osbf_filter_ex(osbf_ctx *ctx, const void *in, void *out, int N, int C, int H, int W, int r, int iters,
                           osbf_dtype dtype, const osbf_options *opts, void *stream);

/*
 * osbf_filter() on HOST buffers: copies `in` to the device, filters, copies the
 * result into `out`, and returns when `out` is filled (synchronous).  The N*C planes
 * go in up to four chunks: a chunk's copies (on two streams owned by the context) overlap
 * the filtering of its neighbours on `stream`.  Pinned host memory gives the fastest
 * copies and the overlap.  The device buffers are owned by the context.
 */
osbf_status osbf_filter_host(osbf_ctx *ctx, const void *in, void *out, int N, int C, int H, int W, int r, int iters,
                             osbf_dtype dtype, void *stream);

/*
 * The fast approximation of Sec. "Fast Approximation to One-sided Box Filter"
 * (Algorithm 3, Eq. (app)), float32, paper tie order, the appendix's boundary.  Per
 * pass one quadrant-mean field (window N1's mean) gives all four quadrant means by
 * shifts of r, and each half window is approximated by the mean of its two quadrant
 * means: N5 ~ (N4+N1)/2, N6 ~ (N3+N2)/2, N7 ~ (N1+N2)/2, N8 ~ (N4+N3)/2; then the
 * selection and update of Algorithm 2.  Not the one-sided box filter itself: its
 * results differ from osbf_filter()'s wherever a half window wins.
 *   in, out   N x C x H x W float32 (device).
 *   maps      optional, as for osbf_filter_ex() (same layout and alignment).
 * Returns OSBF_EINVAL for null pointers, N, C, H or W <= 0, r or iters < 0, in and out
 * overlapping, or unaligned maps; OSBF_EUNSUPPORTED for r > OSBF_MAX_RADIUS.
 */
osbf_status osbf_filter_fast(osbf_ctx *ctx, const float *in, float *out, int N, int C, int H, int W, int r,
                             int iters, uint8_t *maps, void *stream);

/* Largest radius of the 3D filter. */
#define OSBF_MAX_RADIUS_3D 4

/*
 * The 3D one-sided box filter of Sec. "Higher Dimension Case": per voxel the eight
 * corner (octant) windows of (r+1)^3 voxels and the six half windows of (r+1)(2r+1)^2
 * voxels (left/right, down/up, front/back: half along one axis, full along the other
 * two), mean of each, first argmin |mean - U| in the order O1..O8, H9..H14 below, U <-
 * that mean; `iters` passes; volumes replicate-padded by r on every axis once, zeros
 * beyond the padded volume, cropped at the end (the appendix's 2D boundary, extended).
 * Window order: O1..O4 = depth z-r..z with the quadrants N1..N4 of Eq. (6)-(9) in (y, x),
 * O5..O8 = depth z..z+r with N1..N4, H9 = x-r..x, H10 = x..x+r, H11 = y..y+r, H12 =
 * y-r..y, H13 = z-r..z, H14 = z..z+r.  Float32.
 *   in, out   N x C x D x H x W (device).
 *   maps      optional, iters x N*C x (D+2r) x (H+2r) x (W+2r) bytes: window 1..14 per
 *             padded voxel and pass.
 * Returns OSBF_EINVAL for null pointers, non-positive sizes, r or iters < 0, in and out
 * overlapping; OSBF_EUNSUPPORTED for r > OSBF_MAX_RADIUS_3D or volumes whose padded
 * height exceeds 65535 or N*C*(D+2r) exceeds 65535.
 */
osbf_status osbf_filter_3d(osbf_ctx *ctx, const float *in, float *out, int N, int C, int D, int H, int W, int r,
                           int iters, uint8_t *maps, void *stream);

/* Largest radius of the one-sided Gaussian filter. */
#define OSBF_MAX_RADIUS_GAUSS 16

/*
 * The one-sided Gaussian filter: Algorithm 1 with Phi = a weighted mean whose kernels are
 * built as in Sec. "Separable Kernels" from the Gaussian k(u) = exp(-u^2 / (2 sigma^2)),
 * u = -r..r.  Per axis a one-sided kernel k^-/k^+ (distances 0..r from the centre, centre
 * included on both sides, normalised to sum 1) and the full kernel k (normalised over
 * -r..r); window N_i's kernel (windows of Eq. (6)-(13)) is the product of the one-sided
 * kernel on each axis N_i halves and the full kernel on each axis it spans.  First argmin
 * |mean - U| in the order N1..N8, U <- that mean (Algorithm 2's selection), `iters` passes;
 * the appendix's boundary (replicate pad by r once, zeros outside the padded frame with
 * the weights not renormalised there, crop at the end).  sigma = +inf gives flat weights:
 * the one-sided box filter (up to rounding).  Float32.
 *   in, out   N x C x H x W (device).
 *   maps      optional, as for osbf_filter_ex() (same layout and alignment).
 * Returns OSBF_EINVAL for null pointers, N, C, H or W <= 0, r or iters < 0, sigma not > 0,
 * in and out overlapping, unaligned or overlapping maps; OSBF_EUNSUPPORTED for
 * r > OSBF_MAX_RADIUS_GAUSS or N*C > 65535.
 */
osbf_status osbf_filter_gauss(osbf_ctx *ctx, const float *in, float *out, int N, int C, int H, int W, int r,
                              double sigma, int iters, uint8_t *maps, void *stream);

/*
 * Backward (vector-Jacobian product) of the float32 forward, with each pixel's
 * selection frozen to the map stored by the forward (the selection is piecewise
 * constant, so this is the exact gradient wherever no |d_i| tie is crossed).
 * With the selection frozen one pass is linear, U'(p) = (1/n_m(p)) sum_{q in
 * N_m(p) inside the frame} U(q), so its transpose scatters g(p)/n_m(p) over the
 * window; the crop's transpose embeds the gradient into a zero frame and the
 * replicate pad's transpose folds the ring back onto the edge pixels.
 *   grad_out  N x C x H x W float32.      grad_in  N x C x H x W float32 (written).
 *   maps      iters x N*C x (H+2r) rows of osbf_maps_pitch(W, r) uint8, as written by
 *             osbf_filter_ex(); 16-byte aligned (else OSBF_EINVAL).
 */
osbf_status osbf_filter_backward(osbf_ctx *ctx, const float *grad_out, float *grad_in, const uint8_t *maps,
                                 int N, int C, int H, int W, int r, int iters, void *stream);

/* Row pitch, in float32 elements, of the padded frames the library stores
 * (checkpoints): (W + 2r) rounded up to a multiple of 32. */
int osbf_frame_pitch(int W, int r);

/* Row pitch, in bytes, of the selection maps: (W + 2r) rounded up to a multiple of 16
 * (rows start on 16 bytes, so the maps can be written four selections at a time and
 * read back by tensor copies). */
int osbf_maps_pitch(int W, int r);

/*
 * Checkpointed forward / backward (float32): instead of every pass's map, the
 * forward keeps the padded frame before every `interval`-th pass: K = ceil(iters /
 * interval) frames, each N*C x (H+2r) rows of osbf_frame_pitch(W, r) floats (frame k is
 * the state before pass k*interval; frame 0 is the replicate-padded input).  The
 * backward recomputes each segment's selection maps from its checkpoint into context
 * workspace (interval x N*C x (H+2r) x (W+2r) bytes) and back-propagates the segment,
 * last segment first.  Memory: K frames instead of iters maps.
 * Returns OSBF_EINVAL for interval <= 0 and the argument errors of osbf_filter().
 */
osbf_status osbf_filter_checkpointed(osbf_ctx *ctx, const float *in, float *out, float *checkpoints, int interval,
                                     int N, int C, int H, int W, int r, int iters, void *stream);
osbf_status osbf_filter_backward_checkpointed(osbf_ctx *ctx, const float *grad_out, float *grad_in,
                                              const float *checkpoints, int interval, int N, int C, int H, int W,
                                              int r, int iters, void *stream);

/* One image of a batched call: a single H x W float32 plane, its radius and pass count. */
typedef struct {
    const float *in; /* device, H x W */
    float *out;      /* device, H x W */
    int H, W, r, iters;
} osbf_job;

/*
 * Filter `njobs` independent images of different sizes, radii and pass counts in
 * one persistent launch (a device-side queue of (job, fused pass group, tile) items
 * in group-round order; an item starts once its job's previous group has finished),
 * replayed from a CUDA graph that the context caches per job signature (sizes,
 * radii, pass counts and pointers, and the tuned policy, see osbf_autotune_batched()).
 * Equivalent to one osbf_filter() per job (float32, paper tie order), bit for bit with the
 * untuned single-call plan.  Jobs with r = 0 or iters = 0 are copies; jobs with r > 8, and
 * jobs whose tuned single-call choice (osbf_autotune) is another kernel or depth, run as
 * separate filter calls.  Synchronous.
 * Returns OSBF_EINVAL for a bad job (null pointer, non-positive size, in == out),
 * OSBF_ETIMEOUT if a bounded device-side wait gave up (outputs then undefined; the
 * context stays usable).
 */
osbf_status osbf_filter_batched(osbf_ctx *ctx, const osbf_job *jobs, int njobs, void *stream);

/* Tune the batched launch of this job list (synchronous; runs the batch several times): time
 * each layout policy -- the job order within every pass round (as given; by decreasing
 * H x W x passes; or grouped by radius, then by decreasing work, the untuned default) and
 * the resident CTAs per SM (as many as fit, or one fewer) -- each from
 * its own cached graph, and record the fastest for the job signature; later
 * osbf_filter_batched() calls with the same jobs replay that policy's graph.  The policy
 * changes the schedule, never the results. */
osbf_status osbf_autotune_batched(osbf_ctx *ctx, const osbf_job *jobs, int njobs, void *stream);

/* The tuned policy of this job list: *order (0 as given, 1 by decreasing work, 2 grouped by
 * radius, then by decreasing work) and *ctas_per_sm; returns 1 if one is recorded, else 0
 * (the defaults: 2, as many as fit). */
int osbf_batched_policy(osbf_ctx *ctx, const osbf_job *jobs, int njobs, int *order, int *ctas_per_sm);

/* Per-image latency of the last osbf_filter_batched() call: for each job of its
 * persistent launch (jobs with 1 <= r <= 8 and iters >= 1, in job order), the
 * nanoseconds from the first CTA's start to the end of that job's last tile.  Returns
 * the number of values written to ns (at most cap).  Synchronous. */
int osbf_batched_latencies(osbf_ctx *ctx, unsigned long long *ns, int cap);

/* Tune the forward for (dtype, r) on a planes x H x W problem with `iters` passes: time, on
 * the device (synchronous), every candidate -- the tile kernel at each fused depth that fits
 * shared memory and, for float32 (and 8-bit input's float32 passes) at r <= 8, the streaming
 * strip kernel -- on a synthetic non-constant image generated in device memory, and record
 * the fastest {depth, variant} for (dtype, r, the problem's size class: pixels in factors of
 * 4 above 2^20).  Later calls with depth 0 and variant OSBF_VARIANT_AUTO -- plain, map-writing
 * and checkpointed forwards -- use it; the choice is a kernel and a depth, never a change
 * of the filter.  Allocates two scratch images for the duration of the call. */
osbf_status osbf_autotune(osbf_ctx *ctx, osbf_dtype dtype, int planes, int H, int W, int r, int iters);

/* Record a tuned choice without timing (for instance one found on an earlier run):
 * depth 1..OSBF_MAX_DEPTH, variant OSBF_VARIANT_TILE or OSBF_VARIANT_STRIP (depth 1, float32
 * or 8-bit input, r <= 8; else OSBF_EUNSUPPORTED). */
osbf_status osbf_set_tuned(osbf_ctx *ctx, osbf_dtype dtype, int planes, int H, int W, int r, int depth, int variant);

/* The tuned choice recorded for (dtype, r, the size class of planes x H x W): *depth and
 * *variant (osbf_variant); both 0 when nothing was tuned for it. */
osbf_status osbf_tuned(osbf_ctx *ctx, osbf_dtype dtype, int planes, int H, int W, int r, int *depth, int *variant);

/* Synchronise the context's device and report whether any kernel of this context
 * gave up a bounded device-side wait since the last check (OSBF_ETIMEOUT; the
 * outputs of that call are undefined), then clear the record.  OSBF_OK otherwise. */
osbf_status osbf_check(osbf_ctx *ctx);

/* Bound, in nanoseconds, of the batched launch's device-side dependency wait (0 =
 * the default of 2 s).  A smaller bound makes a batched call fail fast with
 * OSBF_ETIMEOUT instead of waiting; it exists so that the timeout path can be
 * exercised without any fault. */
osbf_status osbf_set_wait_timeout(osbf_ctx *ctx, unsigned long long ns);

/* Number of kernel launches the last filter call on `ctx` enqueued. */
int osbf_last_launch_count(const osbf_ctx *ctx);

/*
 * The float32 forward of osbf_filter() without any device allocation.  The paper has
 * no counterpart: this entry point exists for callers that cannot call cudaMalloc,
 * such as real-time pipelines that must not allocate once running (an allocation can
 * synchronise the device or fail under memory pressure) and plug-ins whose host
 * process owns all device memory through its own allocator.
 *   - No context: it runs on the current CUDA device, on `stream`.  The caller passes
 *     device input and output (N x C x H x W float32, not aliasing), as for
 *     osbf_filter(); tie order is the paper's, one pass per launch, with the launch plan
 *     of osbf_filter(): the results equal osbf_filter()'s bit for bit.
 *   - Its scratch is a fixed device array inside the library: two padded frames of at
 *     most OSBF_NOALLOC_MAX_FRAME_FLOATS floats each (N*C*(H+2r) rows of (W+2r) rounded
 *     up to 32 floats); every GPU that loads the library holds this 32 MiB until exit.
 *     Larger problems return OSBF_EUNSUPPORTED, as does r > OSBF_MAX_RADIUS; bad
 *     arguments return OSBF_EINVAL; a failed CUDA call returns OSBF_ECUDA.
 *   - Synchronous: the call reads the kernels' device error word back and returns once
 *     `stream` has finished the filter.  OSBF_ETIMEOUT means a bounded tile-load wait
 *     gave up inside a kernel and the output is undefined.
 *   - The first call on a device looks up the array's device address (once per
 *     device); make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents (each call
 *     rewrites what it reads, and clears the error word).  Calls that overlap on the GPU
 *     race on it: serialise them (one stream, or events).
 */
#define OSBF_NOALLOC_MAX_FRAME_FLOATS (4LL << 20)
osbf_status osbf_filter_noalloc(const float *in, float *out, int N, int C, int H, int W, int r, int iters,
                                void *stream);

/* Library version string. */
const char *osbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OSBF_H */
