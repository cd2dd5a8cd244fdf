/*
 * osbf_oracle.c -- CPU oracle for the One-Sided Box Filter (arxiv 2108.05021).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the library
 * itself never links, imports or calls it, and it shares no code, header or
 * table with the CUDA path.
 *
 * What it computes (paper sections cited per function):
 *   - the eight one-sided windows N1..N8 of Eq. (6)-(13), in frame coordinates
 *     with x = column and y = row (rows increase downward);
 *   - the box kernels k1..k8 of Sec. "One-sided Kernels for Box Filter": a plain
 *     mean over the window, normalised by the full window size n_i (quadrants
 *     (r+1)^2, half windows (r+1)(2r+1)); terms outside the padded frame are zero;
 *   - Algorithm 2: d_i = mean_i - U, m = argmin_i |d_i| (first index in the tie
 *     order wins), U <- U + d_m, all pixels from U^t (Jacobi), for `iters` passes;
 *   - the appendix's boundary: replicate-pad the image by r once, iterate on the
 *     padded frame (its ring evolves too), crop at the end.
 * Arithmetic is FP64 (int64 for the exact 8-bit rule).  Window sums are direct
 * summations over the window, no running sums, no integral images.
 *
 *   - the fast approximation of Sec. "Fast Approximation to One-sided Box Filter"
 *     (Algorithm 3, Eq. (app)): one quadrant-mean field per pass, the other three
 *     quadrants read from it at shifts of r, the four half windows approximated by
 *     the mean of their two quadrant means (oracle_fast_iterate_frame_f64).
 *   - the higher-dimension case of Sec. "Higher Dimension Case" in 3D: eight corner
 *     (octant) windows of (r+1)^3 voxels and six half windows of (r+1)(2r+1)^2 voxels,
 *     the same selection and update (oracle_filter3d_f64).
 *   - the one-sided Gaussian filter (Algorithm 1 with Phi = a weighted mean, Sec.
 *     "Separable Kernels", Eq. (oneside)): the eight windows weighted by products of
 *     normalised one-sided and full 1D Gaussian kernels (oracle_gauss_filter_f64).
 * Readings of the paper taken here (the paper is silent or self-inconsistent):
 *   - `iters` passes (the appendix's `for it = 1:ItNum`), not IterationNum+1;
 *   - tie order "paper": N1..N8; tie order "appendix": the appendix's difference
 *     planes, i.e. N6, N5, N7, N8, N2, N1, N3, N4;
 *   - the updated value is the selected mean itself (U + d_m in exact arithmetic);
 *   - fast approximation: the base field is k_1's mean (window N1: rows y..y+r, cols
 *     x-r..x), so with rows increasing downward the shifts that give N2, N4, N3 are
 *     (0, +r), (-r, 0), (-r, +r) in (row, column); N5 ~ (a4 + a1)/2, N6 ~ (a3 + a2)/2,
 *     N7 ~ (a1 + a2)/2 (the paper's example), N8 ~ (a4 + a3)/2; selection, update,
 *     tie orders and boundary as in Algorithm 2 (the garbled argmin and update lines of
 *     Algorithm 3 read this way);
 *   - 3D: the paper gives no listing and no window order.  Boundary as in 2D (replicate
 *     pad by r once, zeros beyond the padded volume, crop).  Window order: octants O1..O4
 *     = depth z-r..z with the 2D quadrants N1..N4 in (y, x), O5..O8 = depth z..z+r with
 *     N1..N4, then the halves H9 = x-r..x, H10 = x..x+r (full y, z), H11 = y..y+r,
 *     H12 = y-r..y (full x, z), H13 = z-r..z, H14 = z..z+r (full x, y); ties go to the
 *     first window in that order;
 *   - one-sided Gaussian: k(u) = exp(-u^2 / (2 sigma^2)) on -r..r; both one-sided kernels
 *     include the centre tap (Eq. (oneside) writes u > 0 for the right half; the box
 *     kernels and the 3D kernels include u = 0 on both sides, and with it sigma -> inf
 *     gives the one-sided box filter); each 1D kernel is normalised over its own taps,
 *     each 2D window kernel is the product of its two 1D kernels (quadrants: one-sided x
 *     one-sided; halves: one-sided x full); the appendix's boundary (zeros outside the
 *     padded frame, weights not renormalised there).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

/* Storage rounding applied after every iteration (emulates a storage type). */
#define ORACLE_STORE_NONE 0
#define ORACLE_STORE_F32 1
#define ORACLE_STORE_F16 2
#define ORACLE_STORE_BF16 3

/* Window offsets of Eq. (6)-(13).  Index 1..8.  dy = row offset, dx = column offset. */
static void window_offsets(int i, int r, int *dy0, int *dy1, int *dx0, int *dx1) {
    switch (i) {
    case 1: *dx0 = -r; *dx1 = 0; *dy0 = 0;  *dy1 = r; break; /* x-r<=u<=x, y<=v<=y+r   */
    case 2: *dx0 = 0;  *dx1 = r; *dy0 = 0;  *dy1 = r; break; /* x<=u<=x+r, y<=v<=y+r   */
    case 3: *dx0 = 0;  *dx1 = r; *dy0 = -r; *dy1 = 0; break; /* x<=u<=x+r, y-r<=v<=y   */
    case 4: *dx0 = -r; *dx1 = 0; *dy0 = -r; *dy1 = 0; break; /* x-r<=u<=x, y-r<=v<=y   */
    case 5: *dx0 = -r; *dx1 = 0; *dy0 = -r; *dy1 = r; break; /* x-r<=u<=x, |y-v|<=r    */
    case 6: *dx0 = 0;  *dx1 = r; *dy0 = -r; *dy1 = r; break; /* x<=u<=x+r, |y-v|<=r    */
    case 7: *dx0 = -r; *dx1 = r; *dy0 = 0;  *dy1 = r; break; /* |u-x|<=r, y<=v<=y+r    */
    default: *dx0 = -r; *dx1 = r; *dy0 = -r; *dy1 = 0; break; /* 8: |u-x|<=r, y-r<=v<=y */
    }
}

static const int TIE_ORDER[2][8] = {
    {1, 2, 3, 4, 5, 6, 7, 8}, /* paper numbering */
    {6, 5, 7, 8, 2, 1, 3, 4}, /* appendix difference planes 1..8 */
};

/* Window size n_i = number of kernel taps of k_i (fixed, also at the frame edge). */
static long window_count(int i, int r) {
    int dy0, dy1, dx0, dx1;
    window_offsets(i, r, &dy0, &dy1, &dx0, &dx1);
    return (long)(dy1 - dy0 + 1) * (long)(dx1 - dx0 + 1);
}

/* Sum of V over window i around (y, x); pixels outside the FH x FW frame are zero. */
static double window_sum_f64(const double *V, int FH, int FW, int y, int x, int i, int r) {
    int dy0, dy1, dx0, dx1;
    window_offsets(i, r, &dy0, &dy1, &dx0, &dx1);
    int ya = y + dy0, yb = y + dy1, xa = x + dx0, xb = x + dx1;
    if (ya < 0) ya = 0;
    if (yb > FH - 1) yb = FH - 1;
    if (xa < 0) xa = 0;
    if (xb > FW - 1) xb = FW - 1;
    double s = 0.0;
    for (int yy = ya; yy <= yb; ++yy)
        for (int xx = xa; xx <= xb; ++xx) s += V[(size_t)yy * FW + xx];
    return s;
}

static int64_t window_sum_i64(const int64_t *V, int FH, int FW, int y, int x, int i, int r) {
    int dy0, dy1, dx0, dx1;
    window_offsets(i, r, &dy0, &dy1, &dx0, &dx1);
    int ya = y + dy0, yb = y + dy1, xa = x + dx0, xb = x + dx1;
    if (ya < 0) ya = 0;
    if (yb > FH - 1) yb = FH - 1;
    if (xa < 0) xa = 0;
    if (xb > FW - 1) xb = FW - 1;
    int64_t s = 0;
    for (int yy = ya; yy <= yb; ++yy)
        for (int xx = xa; xx <= xb; ++xx) s += V[(size_t)yy * FW + xx];
    return s;
}

/* Round to the nearest value with `mant` fraction bits and minimum normal exponent
 * `emin` (ties to even), i.e. IEEE binary16 (10, -14) or bfloat16 (7, -126).
 * Written from the definition of round-to-nearest-even; no overflow handling is
 * needed for the value ranges used here ([0, 255]). */
static double round_binary(double v, int mant, int emin) {
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    (void)frexp(fabs(v), &e);       /* |v| = f * 2^e, f in [0.5, 1) */
    int lead = e - 1;               /* exponent of the leading bit */
    if (lead < emin) lead = emin;   /* subnormal range: fixed quantum */
    double quantum = ldexp(1.0, lead - mant);
    double q = rint(v / quantum);   /* default rounding mode: nearest, ties to even */
    return q * quantum;
}

double oracle_round_storage(double v, int storage) {
    switch (storage) {
    case ORACLE_STORE_F32: return (double)(float)v;
    case ORACLE_STORE_F16: return round_binary(v, 10, -14);
    case ORACLE_STORE_BF16: return round_binary(v, 7, -126);
    default: return v;
    }
}

void oracle_round_storage_array(double *v, long n, int storage) {
    for (long k = 0; k < n; ++k) v[k] = oracle_round_storage(v[k], storage);
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Replicate padding of one H x W plane into an (H+2r) x (W+2r) frame
 * (the appendix's padarray(..., [r r], 'replicate')). */
void oracle_pad_replicate_f64(const double *in, double *frame, int P, int H, int W, int r) {
    int FH = H + 2 * r, FW = W + 2 * r;
    for (int p = 0; p < P; ++p)
        for (int fy = 0; fy < FH; ++fy) {
            int y = fy - r;
            if (y < 0) y = 0;
            if (y > H - 1) y = H - 1;
            for (int fx = 0; fx < FW; ++fx) {
                int x = fx - r;
                if (x < 0) x = 0;
                if (x > W - 1) x = W - 1;
                frame[((size_t)p * FH + fy) * FW + fx] = in[((size_t)p * H + y) * W + x];
            }
        }
}

/* The crop of the appendix's last line: frame rows/cols r .. r+H-1 / r .. r+W-1. */
void oracle_crop_f64(const double *frame, double *out, int P, int H, int W, int r) {
    int FH = H + 2 * r, FW = W + 2 * r;
    for (int p = 0; p < P; ++p)
        for (int y = 0; y < H; ++y)
            memcpy(&out[((size_t)p * H + y) * W], &frame[((size_t)p * FH + y + r) * FW + r],
                   sizeof(double) * (size_t)W);
}

/* The eight window means at every frame pixel (Eq. (6)-(13) with the box kernels
 * k1..k8): means[(i-1)][p][y][x] = S_i / n_i, zero outside the frame. */
void oracle_window_means_f64(const double *frame, double *means, int P, int FH, int FW, int r) {
    size_t plane = (size_t)FH * FW;
#pragma omp parallel for schedule(static)
    for (long row = 0; row < (long)P * FH; ++row) {
        int p = (int)(row / FH), y = (int)(row % FH);
        const double *V = frame + (size_t)p * plane;
        for (int x = 0; x < FW; ++x)
            for (int i = 1; i <= 8; ++i)
                means[(size_t)(i - 1) * P * plane + (size_t)p * plane + (size_t)y * FW + x] =
                    window_sum_f64(V, FH, FW, y, x, i, r) / (double)window_count(i, r);
    }
}

/*
 * `iters` passes of Algorithm 2 on padded frames, in place.
 *   frame   P x FH x FW, FP64, updated in place.
 *   tie     0 = paper order N1..N8, 1 = appendix order.
 *   maps    optional, iters x P x FH x FW: the selected window index (1..8).
 *   gaps    optional, iters x P x FH x FW: the second-best |d| minus the best |d|,
 *           taken over windows whose mean differs from the selected one (a pixel
 *           whose windows all share one mean gets +inf).
 *   hint    optional, iters x P x FH x FW window indices: the hinted window is taken
 *           instead of this oracle's choice wherever its |d| is within `hint_thresh`
 *           of the best |d| (a near tie); *n_hinted counts the pixels where that
 *           changed the value.
 *   storage rounding applied after every pass (ORACLE_STORE_*).
 */
int oracle_iterate_frame_f64(double *frame, int P, int FH, int FW, int r, int iters, int tie,
                             uint8_t *maps, double *gaps, const uint8_t *hint, double hint_thresh,
                             long long *n_hinted, int storage) {
    if (P <= 0 || FH <= 0 || FW <= 0 || r < 0 || iters < 0 || tie < 0 || tie > 1) return ORACLE_EINVAL;
    size_t plane = (size_t)FH * FW, total = (size_t)P * plane;
    double *next = (double *)malloc(sizeof(double) * (total ? total : 1));
    if (!next) return ORACLE_ENOMEM;
    const int *order = TIE_ORDER[tie];
    long long hinted = 0;
    for (int t = 0; t < iters; ++t) {
#pragma omp parallel for schedule(static) reduction(+ : hinted)
        for (long row = 0; row < (long)P * FH; ++row) {
            int p = (int)(row / FH), y = (int)(row % FH);
            const double *V = frame + (size_t)p * plane;
            for (int x = 0; x < FW; ++x) {
                size_t idx = (size_t)p * plane + (size_t)y * FW + x;
                double u = V[(size_t)y * FW + x];
                double mean[9], ad[9];
                for (int i = 1; i <= 8; ++i) {
                    mean[i] = window_sum_f64(V, FH, FW, y, x, i, r) / (double)window_count(i, r);
                    ad[i] = fabs(mean[i] - u);
                }
                int m = order[0];
                for (int k = 1; k < 8; ++k)
                    if (ad[order[k]] < ad[m]) m = order[k];
                double gap = INFINITY;
                for (int i = 1; i <= 8; ++i)
                    if (i != m && mean[i] != mean[m] && ad[i] - ad[m] < gap) gap = ad[i] - ad[m];
                size_t tidx = (size_t)t * total + idx;
                if (hint) {
                    int h = hint[tidx];
                    if (h >= 1 && h <= 8 && h != m && ad[h] - ad[m] < hint_thresh) {
                        if (mean[h] != mean[m]) hinted += 1;
                        m = h;
                    }
                }
                next[idx] = oracle_round_storage(mean[m], storage);
                if (maps) maps[tidx] = (uint8_t)m;
                if (gaps) gaps[tidx] = gap;
            }
        }
        memcpy(frame, next, sizeof(double) * total);
    }
    free(next);
    if (n_hinted) *n_hinted = hinted;
    return ORACLE_OK;
}

/* The whole filter on P planes of H x W: pad, iterate, crop (the appendix). */
int oracle_filter_f64(const double *in, double *out, int P, int H, int W, int r, int iters, int tie,
                      uint8_t *maps, double *gaps, const uint8_t *hint, double hint_thresh,
                      long long *n_hinted, int storage) {
    if (P <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0) return ORACLE_EINVAL;
    int FH = H + 2 * r, FW = W + 2 * r;
    double *frame = (double *)malloc(sizeof(double) * (size_t)P * FH * FW);
    if (!frame) return ORACLE_ENOMEM;
    oracle_pad_replicate_f64(in, frame, P, H, W, r);
    int st = oracle_iterate_frame_f64(frame, P, FH, FW, r, iters, tie, maps, gaps, hint, hint_thresh,
                                      n_hinted, storage);
    if (st == ORACLE_OK) oracle_crop_f64(frame, out, P, H, W, r);
    free(frame);
    return st;
}

/*
 * The fast approximation (Sec. "Fast Approximation to One-sided Box Filter",
 * Algorithm 3, Eq. (app)), `iters` passes on padded frames, in place.  Per pass:
 *   1. one convolution: D(y, x) = mean of U over N1(y, x) (rows y..y+r, cols x-r..x),
 *      zeros outside the frame, evaluated wherever a lookup below needs it (rows -r..FH-1);
 *   2. the quadrant means by lookup: a1 = D(y, x), a2 = D(y, x+r), a4 = D(y-r, x),
 *      a3 = D(y-r, x+r);
 *   3. the half windows by Eq. (app): a5 = (a4+a1)/2, a6 = (a3+a2)/2, a7 = (a1+a2)/2,
 *      a8 = (a4+a3)/2;
 *   4. d_i = a_i - U, first argmin |d_i| in the tie order, U' = a_m (Jacobi).
 * maps / gaps / hint / n_hinted as in oracle_iterate_frame_f64.
 */
int oracle_fast_iterate_frame_f64(double *frame, int P, int FH, int FW, int r, int iters, int tie, uint8_t *maps,
                                  double *gaps, const uint8_t *hint, double hint_thresh, long long *n_hinted) {
    if (P <= 0 || FH <= 0 || FW <= 0 || r < 0 || iters < 0 || tie < 0 || tie > 1) return ORACLE_EINVAL;
    size_t plane = (size_t)FH * FW, total = (size_t)P * plane;
    /* D on rows -r..FH-1 and columns 0..FW-1+r */
    const int DH = FH + r, DW = FW + r;
    double *next = (double *)malloc(sizeof(double) * (total ? total : 1));
    double *D = (double *)malloc(sizeof(double) * (size_t)P * DH * DW);
    if (!next || !D) {
        free(next);
        free(D);
        return ORACLE_ENOMEM;
    }
    const int *order = TIE_ORDER[tie];
    const double nq = (double)window_count(1, r);
    long long hinted = 0;
    for (int t = 0; t < iters; ++t) {
        /* step 1: the one convolution */
#pragma omp parallel for schedule(static)
        for (long row = 0; row < (long)P * DH; ++row) {
            int p = (int)(row / DH), yy = (int)(row % DH) - r;
            const double *V = frame + (size_t)p * plane;
            for (int x = 0; x < DW; ++x)
                D[(size_t)p * DH * DW + (size_t)(yy + r) * DW + x] = window_sum_f64(V, FH, FW, yy, x, 1, r) / nq;
        }
        /* steps 2-4 */
#pragma omp parallel for schedule(static) reduction(+ : hinted)
        for (long row = 0; row < (long)P * FH; ++row) {
            int p = (int)(row / FH), y = (int)(row % FH);
            const double *V = frame + (size_t)p * plane;
            const double *Dp = D + (size_t)p * DH * DW;
            for (int x = 0; x < FW; ++x) {
                size_t idx = (size_t)p * plane + (size_t)y * FW + x;
                double u = V[(size_t)y * FW + x];
                double a[9], ad[9];
                a[1] = Dp[(size_t)(y + r) * DW + x];           /* D(y, x)     */
                a[2] = Dp[(size_t)(y + r) * DW + x + r];       /* D(y, x+r)   */
                a[4] = Dp[(size_t)y * DW + x];                 /* D(y-r, x)   */
                a[3] = Dp[(size_t)y * DW + x + r];             /* D(y-r, x+r) */
                a[5] = 0.5 * (a[4] + a[1]);
                a[6] = 0.5 * (a[3] + a[2]);
                a[7] = 0.5 * (a[1] + a[2]);
                a[8] = 0.5 * (a[4] + a[3]);
                for (int i = 1; i <= 8; ++i) ad[i] = fabs(a[i] - u);
                int m = order[0];
                for (int k = 1; k < 8; ++k)
                    if (ad[order[k]] < ad[m]) m = order[k];
                double gap = INFINITY;
                for (int i = 1; i <= 8; ++i)
                    if (i != m && a[i] != a[m] && ad[i] - ad[m] < gap) gap = ad[i] - ad[m];
                size_t tidx = (size_t)t * total + idx;
                if (hint) {
                    int h = hint[tidx];
                    if (h >= 1 && h <= 8 && h != m && ad[h] - ad[m] < hint_thresh) {
                        if (a[h] != a[m]) hinted += 1;
                        m = h;
                    }
                }
                next[idx] = a[m];
                if (maps) maps[tidx] = (uint8_t)m;
                if (gaps) gaps[tidx] = gap;
            }
        }
        memcpy(frame, next, sizeof(double) * total);
    }
    free(next);
    free(D);
    if (n_hinted) *n_hinted = hinted;
    return ORACLE_OK;
}

/* The fast approximation on P planes of H x W: pad, iterate, crop (the appendix's boundary). */
int oracle_fast_filter_f64(const double *in, double *out, int P, int H, int W, int r, int iters, int tie,
                           uint8_t *maps, double *gaps, const uint8_t *hint, double hint_thresh,
                           long long *n_hinted) {
    if (P <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0) return ORACLE_EINVAL;
    int FH = H + 2 * r, FW = W + 2 * r;
    double *frame = (double *)malloc(sizeof(double) * (size_t)P * FH * FW);
    if (!frame) return ORACLE_ENOMEM;
    oracle_pad_replicate_f64(in, frame, P, H, W, r);
    int st = oracle_fast_iterate_frame_f64(frame, P, FH, FW, r, iters, tie, maps, gaps, hint, hint_thresh,
                                           n_hinted);
    if (st == ORACLE_OK) oracle_crop_f64(frame, out, P, H, W, r);
    free(frame);
    return st;
}

/*
 * Exact output of one plane on the output rectangle [y0, y1) x [x0, x1), computed
 * from the dependency cone only: each pass widens the region a pixel depends on
 * by r, so after `iters` passes the output there depends only on the frame pixels
 * within iters*r of the rectangle.  Those are padded from `in` and iterated with
 * zeros outside; pixels that the cut edges could affect lie outside the rectangle.
 * `hint` (optional): the selection maps of the whole frame, iters x FH x hint_pitch,
 * applied as in oracle_iterate_frame_f64.
 */
int oracle_filter_region_f64(const double *in, int H, int W, int r, int iters, int tie, int y0, int y1,
                             int x0, int x1, double *out, const uint8_t *hint, int hint_pitch, double hint_thresh,
                             long long *n_hinted) {
    if (H <= 0 || W <= 0 || r < 0 || iters < 0 || y0 < 0 || x0 < 0 || y1 > H || x1 > W || y0 >= y1 ||
        x0 >= x1)
        return ORACLE_EINVAL;
    int FH = H + 2 * r, FW = W + 2 * r;
    long m = (long)iters * r;
    long fy0 = y0 + r - m, fy1 = y1 + r + m, fx0 = x0 + r - m, fx1 = x1 + r + m;
    if (fy0 < 0) fy0 = 0;
    if (fx0 < 0) fx0 = 0;
    if (fy1 > FH) fy1 = FH;
    if (fx1 > FW) fx1 = FW;
    int SH = (int)(fy1 - fy0), SW = (int)(fx1 - fx0);
    double *sub = (double *)malloc(sizeof(double) * (size_t)SH * SW);
    if (!sub) return ORACLE_ENOMEM;
    for (int sy = 0; sy < SH; ++sy) {
        int y = (int)fy0 + sy - r;
        if (y < 0) y = 0;
        if (y > H - 1) y = H - 1;
        for (int sx = 0; sx < SW; ++sx) {
            int x = (int)fx0 + sx - r;
            if (x < 0) x = 0;
            if (x > W - 1) x = W - 1;
            sub[(size_t)sy * SW + sx] = in[(size_t)y * W + x];
        }
    }
    /* optional hints: the full frame's maps (iters x FH x hint_pitch), cut to the sub-frame */
    uint8_t *subhint = NULL;
    if (hint) {
        subhint = (uint8_t *)malloc((size_t)iters * SH * SW + 1);
        if (!subhint) {
            free(sub);
            return ORACLE_ENOMEM;
        }
        for (int t = 0; t < iters; ++t)
            for (int sy = 0; sy < SH; ++sy)
                memcpy(&subhint[((size_t)t * SH + sy) * SW],
                       &hint[((size_t)t * FH + (fy0 + sy)) * (size_t)hint_pitch + fx0], (size_t)SW);
    }
    int st = oracle_iterate_frame_f64(sub, 1, SH, SW, r, iters, tie, NULL, NULL, subhint, hint_thresh, n_hinted,
                                      ORACLE_STORE_NONE);
    free(subhint);
    if (st == ORACLE_OK)
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x)
                out[(size_t)(y - y0) * (x1 - x0) + (x - x0)] =
                    sub[(size_t)(y + r - fy0) * SW + (x + r - fx0)];
    free(sub);
    return st;
}

/*
 * The exact 8-bit rule for the first pass (the appendix casts to single, so the
 * result is FP32): integer window sums S_i, and |mean_i - U| compared exactly by
 * cross-multiplication, |S_i - n_i U| * n_j  vs  |S_j - n_j U| * n_i, in int64.
 * The output is the correctly rounded FP32 value of S_m / n_m (both operands are
 * exact in FP32 for r <= 32, so one IEEE division gives it).
 *   in     P x H x W uint8;  frame_out  P x FH x FW float (the frame after pass 1);
 *   map    optional P x FH x FW selected window index.
 */
int oracle_u8_first_pass(const uint8_t *in, float *frame_out, uint8_t *map, int P, int H, int W, int r,
                         int tie) {
    if (P <= 0 || H <= 0 || W <= 0 || r < 0 || r > 32 || tie < 0 || tie > 1) return ORACLE_EINVAL;
    int FH = H + 2 * r, FW = W + 2 * r;
    size_t plane = (size_t)FH * FW;
    int64_t *V = (int64_t *)malloc(sizeof(int64_t) * (size_t)P * plane);
    if (!V) return ORACLE_ENOMEM;
    for (int p = 0; p < P; ++p)
        for (int fy = 0; fy < FH; ++fy) {
            int y = fy - r;
            if (y < 0) y = 0;
            if (y > H - 1) y = H - 1;
            for (int fx = 0; fx < FW; ++fx) {
                int x = fx - r;
                if (x < 0) x = 0;
                if (x > W - 1) x = W - 1;
                V[(size_t)p * plane + (size_t)fy * FW + fx] = in[((size_t)p * H + y) * W + x];
            }
        }
    const int *order = TIE_ORDER[tie];
#pragma omp parallel for schedule(static)
    for (long row = 0; row < (long)P * FH; ++row) {
        int p = (int)(row / FH), y = (int)(row % FH);
        const int64_t *Vp = V + (size_t)p * plane;
        for (int x = 0; x < FW; ++x) {
            int64_t u = Vp[(size_t)y * FW + x];
            int64_t S[9], n[9], dev[9];
            for (int i = 1; i <= 8; ++i) {
                S[i] = window_sum_i64(Vp, FH, FW, y, x, i, r);
                n[i] = window_count(i, r);
                dev[i] = S[i] - n[i] * u;
                if (dev[i] < 0) dev[i] = -dev[i];
            }
            int m = order[0];
            for (int k = 1; k < 8; ++k) {
                int i = order[k];
                if (dev[i] * n[m] < dev[m] * n[i]) m = i; /* |d_i| < |d_m| exactly */
            }
            size_t idx = (size_t)p * plane + (size_t)y * FW + x;
            frame_out[idx] = (float)S[m] / (float)n[m];
            if (map) map[idx] = (uint8_t)m;
        }
    }
    free(V);
    return ORACLE_OK;
}

/*
 * Transpose (adjoint) of the filter with every selection frozen to `maps`.
 * With m(p) fixed, one pass is linear: U'(p) = (1/n_m(p)) * sum_{q in N_m(p), q in frame} U(q),
 * so its transpose scatters g(p) / n_m(p) to every in-frame q of N_m(p).  The crop's
 * transpose embeds grad_out into a zero frame; the replicate pad's transpose adds each
 * frame pixel's gradient onto the image pixel it was copied from.
 *   grad_out P x H x W, maps iters x P x FH x FW, grad_in P x H x W (written).
 */
int oracle_adjoint_f64(const double *grad_out, const uint8_t *maps, double *grad_in, int P, int H, int W,
                       int r, int iters) {
    if (P <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0) return ORACLE_EINVAL;
    int FH = H + 2 * r, FW = W + 2 * r;
    size_t plane = (size_t)FH * FW, total = (size_t)P * plane;
    double *g = (double *)calloc(total ? total : 1, sizeof(double));
    double *gn = (double *)calloc(total ? total : 1, sizeof(double));
    if (!g || !gn) {
        free(g);
        free(gn);
        return ORACLE_ENOMEM;
    }
    for (int p = 0; p < P; ++p)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                g[(size_t)p * plane + (size_t)(y + r) * FW + (x + r)] = grad_out[((size_t)p * H + y) * W + x];
    for (int t = iters - 1; t >= 0; --t) {
        memset(gn, 0, sizeof(double) * total);
        /* scatter by planes so that planes can run in parallel without races */
#pragma omp parallel for schedule(static)
        for (int p = 0; p < P; ++p) {
            for (int y = 0; y < FH; ++y)
                for (int x = 0; x < FW; ++x) {
                    size_t idx = (size_t)p * plane + (size_t)y * FW + x;
                    int m = maps[(size_t)t * total + idx];
                    int dy0, dy1, dx0, dx1;
                    window_offsets(m, r, &dy0, &dy1, &dx0, &dx1);
                    double w = g[idx] / (double)window_count(m, r);
                    for (int yy = y + dy0; yy <= y + dy1; ++yy) {
                        if (yy < 0 || yy >= FH) continue;
                        for (int xx = x + dx0; xx <= x + dx1; ++xx) {
                            if (xx < 0 || xx >= FW) continue;
                            gn[(size_t)p * plane + (size_t)yy * FW + xx] += w;
                        }
                    }
                }
        }
        double *tmp = g;
        g = gn;
        gn = tmp;
    }
    memset(grad_in, 0, sizeof(double) * (size_t)P * H * W);
    for (int p = 0; p < P; ++p)
        for (int fy = 0; fy < FH; ++fy) {
            int y = fy - r;
            if (y < 0) y = 0;
            if (y > H - 1) y = H - 1;
            for (int fx = 0; fx < FW; ++fx) {
                int x = fx - r;
                if (x < 0) x = 0;
                if (x > W - 1) x = W - 1;
                grad_in[((size_t)p * H + y) * W + x] += g[(size_t)p * plane + (size_t)fy * FW + fx];
            }
        }
    free(g);
    free(gn);
    return ORACLE_OK;
}

/*
 * The 3D one-sided box filter (Sec. "Higher Dimension Case"), `iters` passes on P padded
 * volumes of FD x FH x FW (frames, FP64, updated in place).  Window w = 1..14: offsets
 * [z0,z1] x [y0,y1] x [x0,x1] from the table in window3d(); sums by direct summation with
 * zeros outside the volume; means with the fixed window sizes; first argmin |mean - U|
 * in window order; U' = the chosen mean (Jacobi).  maps / hint as in 2D (14 windows).
 */
static void window3d(int w, int r, int *z0, int *z1, int *y0, int *y1, int *x0, int *x1) {
    /* the 2D quadrants N1..N4 in (y, x): N1 y..y+r, x-r..x; N2 y..y+r, x..x+r;
       N3 y-r..y, x..x+r; N4 y-r..y, x-r..x */
    static const int qy[4][2] = {{0, 1}, {0, 1}, {-1, 0}, {-1, 0}};
    static const int qx[4][2] = {{-1, 0}, {0, 1}, {0, 1}, {-1, 0}};
    if (w <= 8) {
        int q = (w - 1) % 4;
        *z0 = w <= 4 ? -r : 0;
        *z1 = w <= 4 ? 0 : r;
        *y0 = qy[q][0] * r;
        *y1 = qy[q][1] * r;
        *x0 = qx[q][0] * r;
        *x1 = qx[q][1] * r;
        return;
    }
    *z0 = -r; *z1 = r; *y0 = -r; *y1 = r; *x0 = -r; *x1 = r;
    switch (w) {
    case 9: *x1 = 0; break;   /* left  */
    case 10: *x0 = 0; break;  /* right */
    case 11: *y0 = 0; break;  /* down (rows y..y+r) */
    case 12: *y1 = 0; break;  /* up   (rows y-r..y) */
    case 13: *z1 = 0; break;  /* front (depth z-r..z) */
    default: *z0 = 0; break;  /* 14: back (depth z..z+r) */
    }
}

int oracle_filter3d_iterate_f64(double *frame, int P, int FD, int FH, int FW, int r, int iters, uint8_t *maps,
                                const uint8_t *hint, double hint_thresh, long long *n_hinted) {
    if (P <= 0 || FD <= 0 || FH <= 0 || FW <= 0 || r < 0 || iters < 0) return ORACLE_EINVAL;
    size_t vol = (size_t)FD * FH * FW, total = (size_t)P * vol;
    double *next = (double *)malloc(sizeof(double) * (total ? total : 1));
    if (!next) return ORACLE_ENOMEM;
    long long hinted = 0;
    for (int t = 0; t < iters; ++t) {
#pragma omp parallel for schedule(static) reduction(+ : hinted)
        for (long row = 0; row < (long)P * FD * FH; ++row) {
            int p = (int)(row / ((long)FD * FH)), z = (int)((row / FH) % FD), y = (int)(row % FH);
            const double *V = frame + (size_t)p * vol;
            for (int x = 0; x < FW; ++x) {
                size_t idx = (size_t)p * vol + ((size_t)z * FH + y) * FW + x;
                double u = V[((size_t)z * FH + y) * FW + x];
                double mean[15], ad[15];
                for (int w = 1; w <= 14; ++w) {
                    int z0, z1, y0, y1, x0, x1;
                    window3d(w, r, &z0, &z1, &y0, &y1, &x0, &x1);
                    double s = 0.0;
                    for (int zz = z + z0; zz <= z + z1; ++zz) {
                        if (zz < 0 || zz >= FD) continue;
                        for (int yy = y + y0; yy <= y + y1; ++yy) {
                            if (yy < 0 || yy >= FH) continue;
                            for (int xx = x + x0; xx <= x + x1; ++xx)
                                if (xx >= 0 && xx < FW) s += V[((size_t)zz * FH + yy) * FW + xx];
                        }
                    }
                    double n = (double)(z1 - z0 + 1) * (double)(y1 - y0 + 1) * (double)(x1 - x0 + 1);
                    mean[w] = s / n;
                    ad[w] = fabs(mean[w] - u);
                }
                int m = 1;
                for (int w = 2; w <= 14; ++w)
                    if (ad[w] < ad[m]) m = w;
                size_t tidx = (size_t)t * total + idx;
                if (hint) {
                    int h = hint[tidx];
                    if (h >= 1 && h <= 14 && h != m && ad[h] - ad[m] < hint_thresh) {
                        if (mean[h] != mean[m]) hinted += 1;
                        m = h;
                    }
                }
                next[idx] = mean[m];
                if (maps) maps[tidx] = (uint8_t)m;
            }
        }
        memcpy(frame, next, sizeof(double) * total);
    }
    free(next);
    if (n_hinted) *n_hinted = hinted;
    return ORACLE_OK;
}

/* The 3D filter on P volumes of D x H x W: replicate pad by r on every axis, iterate, crop. */
int oracle_filter3d_f64(const double *in, double *out, int P, int D, int H, int W, int r, int iters, uint8_t *maps,
                        const uint8_t *hint, double hint_thresh, long long *n_hinted) {
    if (P <= 0 || D <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0) return ORACLE_EINVAL;
    int FD = D + 2 * r, FH = H + 2 * r, FW = W + 2 * r;
    size_t fvol = (size_t)FD * FH * FW;
    double *frame = (double *)malloc(sizeof(double) * (size_t)P * fvol);
    if (!frame) return ORACLE_ENOMEM;
    for (int p = 0; p < P; ++p)
        for (int z = 0; z < FD; ++z)
            for (int y = 0; y < FH; ++y)
                for (int x = 0; x < FW; ++x) {
                    int sz = z - r < 0 ? 0 : (z - r >= D ? D - 1 : z - r);
                    int sy = y - r < 0 ? 0 : (y - r >= H ? H - 1 : y - r);
                    int sx = x - r < 0 ? 0 : (x - r >= W ? W - 1 : x - r);
                    frame[(size_t)p * fvol + ((size_t)z * FH + y) * FW + x] =
                        in[(((size_t)p * D + sz) * H + sy) * W + sx];
                }
    int st = oracle_filter3d_iterate_f64(frame, P, FD, FH, FW, r, iters, maps, hint, hint_thresh, n_hinted);
    if (st == ORACLE_OK)
        for (int p = 0; p < P; ++p)
            for (int z = 0; z < D; ++z)
                for (int y = 0; y < H; ++y)
                    for (int x = 0; x < W; ++x)
                        out[(((size_t)p * D + z) * H + y) * W + x] =
                            frame[(size_t)p * fvol + ((size_t)(z + r) * FH + y + r) * FW + x + r];
    free(frame);
    return st;
}

/*
 * One-sided Gaussian filter (Algorithm 1 with Phi = the weighted mean of Sec. "Separable
 * Kernels"), `iters` passes on padded frames, in place.  wh[k], k = 0..r: the one-sided
 * 1D kernel (distance k from the centre); wf[k], k = 0..r: the full 1D kernel at offset
 * +-k.  Window i's kernel is wy(dy) * wx(dx) over its offsets (Eq. (6)-(13)), with wy / wx
 * = wh on a one-sided axis and wf on a full axis.  Selection and update as Algorithm 2.
 */
int oracle_gauss_iterate_frame_f64(double *frame, int P, int FH, int FW, int r, int iters, int tie,
                                   double sigma, uint8_t *maps, const uint8_t *hint, double hint_thresh,
                                   long long *n_hinted) {
    if (P <= 0 || FH <= 0 || FW <= 0 || r < 0 || iters < 0 || tie < 0 || tie > 1 || !(sigma > 0))
        return ORACLE_EINVAL;
    double *g = (double *)malloc(sizeof(double) * (r + 1));
    double *wh = (double *)malloc(sizeof(double) * (r + 1));
    double *wf = (double *)malloc(sizeof(double) * (r + 1));
    size_t plane = (size_t)FH * FW, total = (size_t)P * plane;
    double *next = (double *)malloc(sizeof(double) * (total ? total : 1));
    if (!g || !wh || !wf || !next) {
        free(g); free(wh); free(wf); free(next);
        return ORACLE_ENOMEM;
    }
    double sh = 0.0, sf = 0.0;
    for (int k = 0; k <= r; ++k) {
        g[k] = exp(-(double)k * k / (2.0 * sigma * sigma));
        sh += g[k];
        sf += k == 0 ? g[k] : 2.0 * g[k];
    }
    for (int k = 0; k <= r; ++k) {
        wh[k] = g[k] / sh;
        wf[k] = g[k] / sf;
    }
    const int *order = TIE_ORDER[tie];
    long long hinted = 0;
    for (int t = 0; t < iters; ++t) {
#pragma omp parallel for schedule(static) reduction(+ : hinted)
        for (long row = 0; row < (long)P * FH; ++row) {
            int p = (int)(row / FH), y = (int)(row % FH);
            const double *V = frame + (size_t)p * plane;
            for (int x = 0; x < FW; ++x) {
                size_t idx = (size_t)p * plane + (size_t)y * FW + x;
                double u = V[(size_t)y * FW + x];
                double mean[9], ad[9];
                for (int i = 1; i <= 8; ++i) {
                    int dy0, dy1, dx0, dx1;
                    window_offsets(i, r, &dy0, &dy1, &dx0, &dx1);
                    const int yfull = dy0 == -r && dy1 == r, xfull = dx0 == -r && dx1 == r;
                    double s = 0.0;
                    for (int dy = dy0; dy <= dy1; ++dy) {
                        int yy = y + dy;
                        if (yy < 0 || yy >= FH) continue;
                        double wy = yfull ? wf[abs(dy)] : wh[abs(dy)];
                        for (int dx = dx0; dx <= dx1; ++dx) {
                            int xx = x + dx;
                            if (xx < 0 || xx >= FW) continue;
                            double wx = xfull ? wf[abs(dx)] : wh[abs(dx)];
                            s += wy * wx * V[(size_t)yy * FW + xx];
                        }
                    }
                    mean[i] = s;
                    ad[i] = fabs(s - u);
                }
                int m = order[0];
                for (int k = 1; k < 8; ++k)
                    if (ad[order[k]] < ad[m]) m = order[k];
                size_t tidx = (size_t)t * total + idx;
                if (hint) {
                    int h = hint[tidx];
                    if (h >= 1 && h <= 8 && h != m && ad[h] - ad[m] < hint_thresh) {
                        if (mean[h] != mean[m]) hinted += 1;
                        m = h;
                    }
                }
                next[idx] = mean[m];
                if (maps) maps[tidx] = (uint8_t)m;
            }
        }
        memcpy(frame, next, sizeof(double) * total);
    }
    free(g); free(wh); free(wf); free(next);
    if (n_hinted) *n_hinted = hinted;
    return ORACLE_OK;
}

/* The one-sided Gaussian filter on P planes of H x W: pad, iterate, crop. */
int oracle_gauss_filter_f64(const double *in, double *out, int P, int H, int W, int r, int iters, int tie,
                            double sigma, uint8_t *maps, const uint8_t *hint, double hint_thresh,
                            long long *n_hinted) {
    if (P <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0) return ORACLE_EINVAL;
    int FH = H + 2 * r, FW = W + 2 * r;
    double *frame = (double *)malloc(sizeof(double) * (size_t)P * FH * FW);
    if (!frame) return ORACLE_ENOMEM;
    oracle_pad_replicate_f64(in, frame, P, H, W, r);
    int st = oracle_gauss_iterate_frame_f64(frame, P, FH, FW, r, iters, tie, sigma, maps, hint, hint_thresh,
                                            n_hinted);
    if (st == ORACLE_OK) oracle_crop_f64(frame, out, P, H, W, r);
    free(frame);
    return st;
}
