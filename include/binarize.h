/*
 * binarize.h — C ABI of the GB300 local adaptive binarization library.
 *
 * The library computes, for every pixel (i, j) of an 8-bit gray image, the
 * statistics of the h x w window around it and compares the pixel with a
 * local threshold, as in Chan, "Memory-efficient and fast implementation of
 * local adaptive binarization methods" (arXiv 1905.13038):
 *
 *   window     rows (i-o, i+u], columns (j-l, j+r] with l = floor((w+1)/2),
 *              r = floor(w/2), o = floor((h+1)/2), u = floor(h/2)
 *              (Algorithm 1, Sec. 1 definitions of m and s);
 *   border     pixels outside the image count as 0 and n is the number of
 *              in-image window pixels (Sec. 3.2 assumptions, Algorithm 1);
 *   sums       S1 = sum I, S2 = sum I^2, exact integers (Sec. 3.1, Sec. 3.3);
 *   threshold  Sauvola t = m (1 + k (s/R - 1)) (Sec. 1, Table 1),
 *              Niblack t = m + k s (Table 1), with m = S1/n and
 *              s = sqrt(V)/n, V = n S2 - S1^2 (exact 64-bit integer);
 *              local quantile t = Q - offset (Sec. 3.4);
 *   output     bit 0 where I <= t (dark, foreground), 1 elsewhere
 *              (Algorithm 1), packed LSB first: bit (j & 7) of byte (j >> 3)
 *              of each output row; padding bits of the last byte are 0.
 *
 * Floating point.  The reference threshold is the "canonical" FP64
 * evaluation, every operation IEEE binary64 round-to-nearest without FMA
 * contraction, in exactly this order:
 *     nd = n; m = S1/nd; s = sqrt(V/(nd*nd));
 *     Sauvola t = m*(1 + k*(s/R - 1));  Niblack t = m + k*s.
 * BZ_FP64 reproduces its decisions bit for bit; BZ_FP32 evaluates the same
 * formula in FP32 and may differ on pixels within ~1e-4 gray levels of t.
 *
 * Memory.  Every image/output pointer is a DEVICE pointer owned by the
 * caller (for instance a torch tensor); the library neither frees nor keeps
 * it past the completion of the work on `stream` (a cudaStream_t passed as
 * void*, NULL = legacy default stream).  The image has H rows of in_pitch
 * >= W bytes, all H * in_pitch of them readable: the kernels may read a row's
 * bytes past column W (never using them) when they load aligned 8-byte words.
 * out has H rows of out_pitch >= ceil(W/8) bytes.  Only the first ceil(W/8)
 * bytes of each output row are written.  Image and output
 * must not overlap (Sec. 3.2 assumptions): overlap -> BZ_EOVERLAP.
 * The library's own stream-ordered scratch (stripe sums of tall windows,
 * global statistics, in-place bands) comes from a memory pool per device
 * that keeps up to 256 MB between calls ("the library's pool"), or, on a
 * capturing stream, from the graph's own allocations.
 *
 * Errors.  Argument errors are reported synchronously and nothing is
 * launched.  Launch failures return BZ_ECUDA.  Work is asynchronous with
 * respect to the host; kernel-side faults surface at the caller's next
 * synchronisation.  No entry point aborts the process.
 *
 * Limits: 1 <= H, W <= 2^31 - 1; 1 <= h, w <= 511 (keeps V < 2^53 so the
 * FP64 threshold sees it exactly).
 */
#ifndef BINARIZE_H
#define BINARIZE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BZ_OK = 0,
    BZ_EINVAL = 1,          /* bad argument (size, pitch, window, parameter) */
    BZ_EOVERLAP = 2,        /* image and output buffers overlap              */
    BZ_ENOMEM = 3,          /* the library could not allocate its scratch    */
    BZ_EBUDGET = 4,         /* server: request larger than the HBM budget    */
    BZ_ECUDA = 5,           /* a CUDA call or kernel launch failed           */
    BZ_ETIMEOUT = 6,        /* server: wait timed out (request cancelled)    */
    BZ_EDEVICE_TIMEOUT = 7, /* a bounded device-side wait gave up            */
    BZ_ECANCELLED = 8       /* server: request cancelled                     */
} bz_status;

typedef enum {
    BZ_FP64 = 0,        /* decisions identical to the canonical FP64 threshold:
                           certified FP32 filter + FP64 for near-ties         */
    BZ_FP32 = 1,        /* FP32 threshold only (fast, may flip near-ties)    */
    BZ_FP64_DIRECT = 2  /* canonical FP64 threshold evaluated for every pixel */
} bz_precision;

typedef enum {
    BZ_SAUVOLA = 0,
    BZ_NIBLACK = 1,
    BZ_QUANTILE = 2,
    BZ_WOLF = 3,
    BZ_FENG = 4,
    BZ_RAIS = 5,
    BZ_NICK = 6,
    BZ_PHANSALKAR = 7
} bz_method;

/* Human-readable name of a status code (static string, never NULL). */
const char *bz_status_string(bz_status s);

/* Sauvola binarization (Sec. 1 formula; Algorithm 1; sqrt-free identity of
 * Sec. 3.2 for k >= 0).  k: any finite value (the paper requires k >= 0 for
 * its square-root-free form; the library accepts any k); R > 0 finite. */
bz_status binarize_sauvola(const uint8_t *image, int64_t H, int64_t W,
                           int64_t in_pitch, int32_t h, int32_t w, double k,
                           double R, uint8_t *out, int64_t out_pitch,
                           bz_precision precision, void *stream);

/* Niblack binarization, t = m + k s (Table 1).  k: any finite value. */
bz_status binarize_niblack(const uint8_t *image, int64_t H, int64_t W,
                           int64_t in_pitch, int32_t h, int32_t w, double k,
                           uint8_t *out, int64_t out_pitch,
                           bz_precision precision, void *stream);

/* Local-quantile binarization (Sec. 3.4, sliding histograms).
 * Q = rho-th smallest gray level of the clipped window with
 * rho = max(1, ceil(n * q_num / q_den)) computed in integers
 * (q = 1/2 gives the lower median); bit = 0 iff I <= Q - offset.
 * 0 <= q_num <= q_den, q_den >= 1, |offset| <= 255. */
bz_status binarize_quantile(const uint8_t *image, int64_t H, int64_t W,
                            int64_t in_pitch, int32_t h, int32_t w,
                            int32_t q_num, int32_t q_den, int32_t offset,
                            uint8_t *out, int64_t out_pitch, void *stream);

/* Parity export of the exact window statistics (Sec. 1 definitions computed
 * with the Sec. 3.1 recursive identities): S1, S2 and n as dense H x W
 * row-major device arrays (uint32, uint64, uint32).  Any of the three may
 * be NULL to skip it. */
bz_status window_sums(const uint8_t *image, int64_t H, int64_t W,
                      int64_t in_pitch, int32_t h, int32_t w, uint32_t *S1,
                      uint64_t *S2, uint32_t *n, void *stream);

/* Parity export of the window quantile Q (Sec. 3.4): dense H x W uint8. */
bz_status window_quantile(const uint8_t *image, int64_t H, int64_t W,
                          int64_t in_pitch, int32_t h, int32_t w,
                          int32_t q_num, int32_t q_den, uint8_t *Q,
                          void *stream);

/* FP32-versus-FP64 report for a Sauvola (method 0) or Niblack (method 1)
 * configuration: adds to *flips_dev the number of pixels whose BZ_FP32
 * decision differs from the canonical FP64 decision, and raises
 * *max_abs_dt_dev to the largest |t32 - t64| seen.  Both are caller-owned
 * device scalars (initialise them to 0).  R is ignored for Niblack. */
bz_status binarize_precision_report(int32_t method, const uint8_t *image,
                                    int64_t H, int64_t W, int64_t in_pitch,
                                    int32_t h, int32_t w, double k, double R,
                                    uint64_t *flips_dev,
                                    double *max_abs_dt_dev, void *stream);

/* Number of kernels one binarize_sauvola / binarize_niblack call on an
 * H x W image with an h x w window launches on the current device (the
 * window kernel, plus the stripe pre-pass for tall windows: it depends on the
 * device's SM count).  For planning graph captures and for counting launches;
 * -1 for invalid arguments. */
int32_t bz_kernels_per_call(int64_t H, int64_t W, int32_t h, int32_t w,
                            bz_precision precision);

/* The window kernel's tile schedule for an H x W image on a GPU with `sms`
 * SMs, computed on the host without a device (pure arithmetic; for planning
 * and tests).  pipe: the pipelined kernel (else the generic one); stripes:
 * the launch starts from the stripe pre-pass.  Writes out[0..5] = tile
 * columns (256 pixels each), interior tile rows, edge tile rows, edge tiles
 * (listed first, alternating the first and last tile column), tiles in total
 * and the warps resident at once (one wave).  Returns 0, or -1 for invalid
 * arguments. */
int32_t bz_tile_schedule(int64_t H, int64_t W, int32_t sms, int32_t pipe,
                         int32_t stripes, int64_t *out);

/* Number of pixels the most recent BZ_FP64 call on this device could not
 * decide in FP32 and evaluated in FP64, read back synchronously after the
 * stream finishes (0 before any BZ_FP64 call).  Single-image calls count into
 * two per-device counters in turn, each zeroed by the call after it, so the
 * count is that of the latest call only while calls on the device are
 * ordered (one stream); batches count into a third.  Diagnostic only;
 * returns -1 when unknown. */
int64_t bz_last_fp64_fallbacks(void *stream);

/* Sauvola (method 0) or Niblack (method 1) from HOST memory: the image is
 * uploaded, binarized and the packed output downloaded.  The call returns once
 * the work is enqueued; every later operation on `stream` (and a synchronize
 * of it) comes after the download, so synchronise the stream before reading
 * out_host.  The call does not wait for work already on `stream`: the host
 * image is read from the moment of the call.  image_host: H rows of
 * in_pitch >= W bytes; out_host: H rows of out_pitch >= ceil(W/8) bytes; both
 * must stay valid and the image unchanged until the stream has been
 * synchronised, and they must not overlap.  Page-locked (pinned) host memory
 * makes the copies asynchronous; pageable memory works but the copies then
 * block the host.  The library runs the upload, compute and download of a
 * device's calls on three streams of its own with two sets of device buffers
 * used in turn (grown with cudaMalloc when a larger page arrives, after the
 * set's previous call is done), so that a sequence of calls overlaps one
 * call's upload and download with its neighbours' compute.  Calls from
 * several host threads are serialised on a per-device lock while they
 * enqueue.  CUDA failure -> BZ_ECUDA (nothing of the call is then left in
 * flight).  Results equal binarize_sauvola / binarize_niblack. */
bz_status binarize_host(int32_t method, const uint8_t *image_host, int64_t H,
                        int64_t W, int64_t in_pitch, int32_t h, int32_t w,
                        double k, double R, uint8_t *out_host,
                        int64_t out_pitch, bz_precision precision,
                        void *stream);

/* The same for n window sizes of one image (multi-scale use): the image is
 * uploaded once, binarized with each window (h[q], w[q]) in turn and the n
 * packed outputs downloaded into out_host[q] (each H rows of out_pitch
 * bytes; none may overlap the image or one another).  1 <= n <= 64; h, w
 * and out_host are host arrays of n entries, read during the call only.
 * bz_last_fp64_fallbacks then reports the sum over the n windows.  Ordering,
 * lifetime and errors as for binarize_host. */
bz_status binarize_host_multi(int32_t method, const uint8_t *image_host,
                              int64_t H, int64_t W, int64_t in_pitch,
                              int32_t n, const int32_t *h, const int32_t *w,
                              double k, double R, uint8_t *const *out_host,
                              int64_t out_pitch, bz_precision precision,
                              void *stream);

/* ---------------------------------------------------------------------- */
/* In-place binarization (Sec. 3.2 assumptions: the algorithm can be made */
/* in-place by keeping the gray levels that later windows still need).    */
/* ---------------------------------------------------------------------- */

/* Sauvola (method 0) or Niblack (method 1) written over the image itself:
 * on return row i of `image` starts with its ceil(W/8) packed output bytes
 * (same bit layout as binarize_sauvola); the bytes after them keep their
 * gray levels.  The image is processed in bands of band_rows rows (0 picks
 * max(o, 256)); band k goes to a library scratch of two bands
 * (2 * band_rows * ceil(W/8) bytes, stream-ordered, from the library's pool) and is
 * copied into place after band k+1 has read its rows, which needs
 * band_rows >= o = floor((h+1)/2) (else BZ_EINVAL).  Results equal
 * binarize_sauvola / binarize_niblack with a separate output.  Smaller
 * bands use less memory and run more, smaller launches. */
bz_status binarize_inplace(int32_t method, uint8_t *image, int64_t H, int64_t W,
                           int64_t pitch, int32_t h, int32_t w, double k,
                           double R, int64_t band_rows, bz_precision precision,
                           void *stream);

/* Scratch bytes binarize_inplace takes for these sizes (-1 if invalid), for
 * admission under a memory budget. */
int64_t bz_inplace_scratch_bytes(int64_t H, int64_t W, int32_t h, int64_t band_rows);

/* The same result with the axes exchanged (Sec. 3.3: the roles of H and W
 * swap, so the scratch follows H instead of W): the image is processed in
 * bands of band_cols columns (0 picks the smallest allowed: 256 for
 * w <= 450, else 512; otherwise a multiple of 256 at least that), each over
 * all H rows.  Band k's packed bits go to a library scratch of one band
 * (H * band_cols / 8 bytes, or H * ceil(W/8) if W is smaller;
 * stream-ordered, from the library's pool) and are copied into bytes
 * [c0/8, ceil(c1/8)) of every row right after the band: columns left of
 * c1/8 are read by no later band because 7 c1 / 8 >= l - 1.  Arguments,
 * layout and errors as binarize_inplace (BZ_EINVAL for a band_cols that is
 * not allowed).  Each band is a narrow launch, so this is slower than
 * binarize_inplace; it takes less scratch when H * band_cols / 8 is below
 * 2 * max(o, 256) * ceil(W/8), which with the default bands means H < 2 W
 * (w <= 450) or H < W (wider windows) for images taller than 256 rows. */
bz_status binarize_inplace_cols(int32_t method, uint8_t *image, int64_t H,
                                int64_t W, int64_t pitch, int32_t h, int32_t w,
                                double k, double R, int64_t band_cols,
                                bz_precision precision, void *stream);

/* Scratch bytes binarize_inplace_cols takes (-1 if invalid). */
int64_t bz_inplace_cols_scratch_bytes(int64_t H, int64_t W, int32_t w,
                                      int64_t band_cols);

/* ---------------------------------------------------------------------- */
/* Local minimum and maximum (Sec. 3.4: Bernsen's midrange and the local  */
/* contrast, kept recursively).  The window is Algorithm 1's, clipped to  */
/* the image; pixels outside the image take no part (they are neither a   */
/* minimum nor a maximum), so every window holds at least its own centre.  */
/* ---------------------------------------------------------------------- */

/* Parity export: mn and mx, dense H x W uint8 device arrays (caller-owned,
 * neither overlapping the image nor each other). */
bz_status window_minmax(const uint8_t *image, int64_t H, int64_t W,
                        int64_t in_pitch, int32_t h, int32_t w, uint8_t *mn,
                        uint8_t *mx, void *stream);

/* Bernsen binarization, in integers: with c = mx - mn,
 *   c >= contrast_limit:  bit = 0 iff 2 I <= mn + mx   (I <= midrange);
 *   c <  contrast_limit:  the window is one class, bit = 0 iff
 *                         mn + mx <= 255 (its midrange is dark).
 * 0 <= contrast_limit <= 256 (0: midrange everywhere; 256: never). */
bz_status binarize_bernsen(const uint8_t *image, int64_t H, int64_t W,
                           int64_t in_pitch, int32_t h, int32_t w,
                           int32_t contrast_limit, uint8_t *out,
                           int64_t out_pitch, void *stream);

/* ---------------------------------------------------------------------- */
/* Haar-like window sums (Sec. 3.4: the recursive sums replace integral   */
/* images for Haar-like features).  For every pixel (i, j) the sum over   */
/* Algorithm 1's h x w window of f(a) g(b) I(i-o+1+a, j-l+1+b), where the  */
/* window's rows are cut into n_row segments (row_len[s] rows of weight    */
/* row_wt[s], top to bottom) and its columns into n_col segments (left to  */
/* right); h = sum row_len, w = sum col_len.  Pixels outside the image are */
/* 0.  Viola and Jones's features: two segments of weights +1/-1 in one    */
/* direction (edge), three of -1/+2/-1 (line), two by two (diagonal).      */
/* The cost per pixel depends on the number of segments, not on h or w.    */
/* ---------------------------------------------------------------------- */
typedef struct {
    int32_t n_row, n_col;          /* 1..4 each                            */
    int32_t row_len[4], row_wt[4]; /* lengths >= 1, weights in [-127, 127] */
    int32_t col_len[4], col_wt[4];
} bz_haar;

/* out: dense H x W int32 device array (caller-owned, not overlapping the
 * image).  Limits: 1 <= h, w <= 511 and 255 h w max|row_wt| max|col_wt|
 * < 2^31 (so the result is exact); otherwise BZ_EINVAL.  `feature` is a
 * host pointer, read during the call. */
bz_status haar_feature(const uint8_t *image, int64_t H, int64_t W,
                       int64_t in_pitch, const bz_haar *feature, int32_t *out,
                       void *stream);

/* ---------------------------------------------------------------------- */
/* The other Table 1 methods (Sec. 3.4: one changed condition on the same */
/* window statistics).  L, M and S are the global minimum, mean and        */
/* population standard deviation of the image (Table 1 notations), found   */
/* by one reduction pass on `stream` before the window pass.  The library  */
/* takes 24 bytes of stream-ordered scratch (library pool) per call and   */
/* frees it on the stream: allocation failure -> BZ_ENOMEM.                */
/*                                                                        */
/* Canonical FP64 thresholds (every operation binary64 round-to-nearest,   */
/* no contraction, in this order; m, s, V as above, nd = n):               */
/*   Wolf        t = m - (k*(m - L)) * (1 - s/R)                           */
/*   Feng        x = s/R;  t = (alpha1*m + (k1*pow(x, 1+gamma))*(m - L))   */
/*                             + (k2*pow(x, gamma))*L                      */
/*   Rais        d = max(m*s, M*S);  f = d > 0 ? (m*s - M*S)/d : 0;        */
/*               t = m + (k*f)*s                                           */
/*   NICK        t = m + k*sqrt(V/(nd*nd) + (m*m)*((nd - 1)/nd))           */
/*               (Table 1's window area hw is the clipped count n)          */
/*   Phansalkar  t = m * ((1 + p*exp(-(q*m))) + k*(s/R - 1))               */
/* with L = min I, M = sum/N, S = sqrt(Vg/(N*N)), Vg = N*sumsq - sum^2     */
/* exact (128-bit) and rounded once to double.  Feng and Phansalkar use    */
/* the device pow/exp, which may differ from another libm by an ulp, so    */
/* their decisions can differ from another implementation only where       */
/* |I - t| is a few ulps of t.  The precision modes are those of Sauvola:  */
/* BZ_FP64 (certified FP32 + FP64 near-ties), BZ_FP32, BZ_FP64_DIRECT.     */
/*                                                                        */
/* Parameters: finite, |x| <= 1e6; R in [1e-6, 1e9]; Feng gamma in [0, 16];*/
/* Phansalkar q >= 0 (on gray levels 0..255: the published normalised     */
/* setting p = 2, q = 10, k = 0.25, R = 0.5 is q = 10/255, R = 127.5 here).*/
/* Image limit for these methods: H*W <= 2^44.                             */
/* ---------------------------------------------------------------------- */
bz_status binarize_wolf(const uint8_t *image, int64_t H, int64_t W,
                        int64_t in_pitch, int32_t h, int32_t w, double k,
                        double R, uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream);

/* Feng (Table 1 form): alpha1 multiplies m directly. */
bz_status binarize_feng(const uint8_t *image, int64_t H, int64_t W,
                        int64_t in_pitch, int32_t h, int32_t w, double alpha1,
                        double k1, double k2, double gamma, double R,
                        uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream);

/* Rais (Table 1 prints k = 0.3). */
bz_status binarize_rais(const uint8_t *image, int64_t H, int64_t W,
                        int64_t in_pitch, int32_t h, int32_t w, double k,
                        uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream);

/* NICK (Khurshid et al.), k typically in [-0.2, -0.1]. */
bz_status binarize_nick(const uint8_t *image, int64_t H, int64_t W,
                        int64_t in_pitch, int32_t h, int32_t w, double k,
                        uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream);

bz_status binarize_phansalkar(const uint8_t *image, int64_t H, int64_t W,
                              int64_t in_pitch, int32_t h, int32_t w,
                              double k, double R, double p, double q,
                              uint8_t *out, int64_t out_pitch,
                              bz_precision precision, void *stream);

/* Parity export of the global statistics: stats_dev[0..2] = (L, M, S) as
 * doubles, sums_dev[0..2] = (sum I, sum I^2, N) (sums_dev may be NULL);
 * both caller-owned device arrays.  H*W <= 2^44. */
bz_status global_stats(const uint8_t *image, int64_t H, int64_t W,
                       int64_t in_pitch, double *stats_dev, uint64_t *sums_dev,
                       void *stream);

/* FP32-versus-FP64 report for any Table 1 method (bz_method other than
 * BZ_QUANTILE).  params: HOST array of 8 doubles {k, R, alpha1, k1, k2,
 * gamma, p, q} (unused entries ignored).  Semantics as
 * binarize_precision_report. */
bz_status binarize_precision_report_ext(int32_t method, const uint8_t *image,
                                        int64_t H, int64_t W, int64_t in_pitch,
                                        int32_t h, int32_t w,
                                        const double *params,
                                        uint64_t *flips_dev,
                                        double *max_abs_dt_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Batched execution: many images of uneven sizes in one launch.          */
/* ---------------------------------------------------------------------- */
typedef struct {
    const uint8_t *image; /* device */
    uint8_t *out;         /* device */
    int64_t H, W, in_pitch, out_pitch;
    int32_t h, w;
    int32_t method;       /* bz_method */
    double k, R;          /* Sauvola / Niblack parameters */
    int32_t q_num, q_den, offset; /* quantile parameters */
} bz_job;

/* Runs n jobs (host array, copied before return) as one persistent launch
 * over a device work list.  precision applies to Sauvola/Niblack jobs.
 * Every job is validated first; on any invalid job nothing is launched and
 * BZ_EINVAL/BZ_EOVERLAP is returned. */
bz_status binarize_batch(const bz_job *jobs_host, int32_t n,
                         bz_precision precision, void *stream);

/* Allocation-free variant of binarize_batch.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory at call time,
 * such as services that reserve all of the GPU's memory up front in their own
 * arena or caching allocator (a library cudaMalloc would fail or fragment
 * their pool) and latency-critical loops that must not wait on the driver's
 * allocator.  It runs the same persistent kernels as binarize_batch, with
 * identical results, but its device work list lives in one fixed array that
 * is part of the library image (about 150 KB, held by every GPU that loads
 * the library until the process exits), and it calls no allocation routine.
 *   - n <= BZ_NOALLOC_MAX_JOBS; larger n returns BZ_EINVAL, nothing launched.
 *   - The array is placed on a device when the library's CUDA module is
 *     loaded there.  Under CUDA's default lazy module loading that happens at
 *     the first call on the device (which also looks up the array's device
 *     address with cudaGetSymbolAddress and sets the kernels' attributes), so
 *     a caller that reserves all of its device memory afterwards must make
 *     one call, or any other library call, first; with
 *     CUDA_MODULE_LOADING=EAGER the array is placed when the context is
 *     created.  Later calls place nothing and allocate nothing.
 *   - Not for stream capture: each call stages the work list in one static
 *     host buffer that the next call overwrites, so a captured copy would
 *     replay another call's list.  A call on a capturing stream returns
 *     BZ_EINVAL and enqueues nothing.
 *   - Every call on a device shares the one work list: calls whose work
 *     overlaps on the GPU (for instance on two streams) race and corrupt each
 *     other's list.  Order them on one stream or synchronise in between.
 *   - jobs_host is read before the call returns; the copy to the device is
 *     ordered on `stream`.  Argument errors are reported synchronously. */
#define BZ_NOALLOC_MAX_JOBS 512
bz_status binarize_batch_noalloc(const bz_job *jobs_host, int32_t n,
                                 bz_precision precision, void *stream);

/* ---------------------------------------------------------------------- */
/* Served execution: continuous batching of requests on the device.       */
/* ---------------------------------------------------------------------- */
typedef struct bz_server bz_server;

/* hbm_budget_bytes: upper bound on the summed device bytes of the requests
 * in flight (image + output for a job with a separate output; image + the
 * in-place scratch for an in-place job, below); max_slots: requests in
 * flight at most.
 * In-place requests: a Sauvola or Niblack job with out == image and
 * out_pitch == in_pitch is binarized over its image as binarize_inplace does
 * (binarize_batch rejects such a job with BZ_EOVERLAP).  It is admitted with
 * row bands (binarize_inplace, scratch bz_inplace_scratch_bytes(H, W, h, 0))
 * when image + that scratch fits the budget left, else with column bands
 * (binarize_inplace_cols, scratch bz_inplace_cols_scratch_bytes(H, W, w, 0))
 * when those fit; otherwise it waits at the head of the queue.  Submission
 * returns BZ_EBUDGET when image + the smaller scratch exceeds the budget. */
bz_status bz_server_create(int64_t hbm_budget_bytes, int32_t max_slots,
                           bz_server **out);
/* Queues a job; its buffers must stay valid until bz_server_wait returns
 * BZ_OK or BZ_ECANCELLED for the ticket, or BZ_ETIMEOUT for a request that
 * had not started (see bz_server_wait). */
bz_status bz_server_submit(bz_server *srv, const bz_job *job,
                           bz_precision precision, uint64_t *ticket);
/* Waits for a ticket; timeout_ms < 0 waits forever.  Returns the request's
 * status (and forgets the ticket) when it finished within the timeout.
 * Otherwise BZ_ETIMEOUT, without waiting further: a request that had not
 * started is dropped and its buffers are free; a request already running
 * cannot be recalled from the GPU, so it is cancelled but keeps its ticket,
 * and its buffers stay in use until a later bz_server_wait on the same ticket
 * returns BZ_ECANCELLED (a wait may time out again meanwhile) or until
 * bz_server_destroy returns. */
bz_status bz_server_wait(bz_server *srv, uint64_t ticket, int32_t timeout_ms);
bz_status bz_server_cancel(bz_server *srv, uint64_t ticket);
/* Cancels queued requests, waits for the in-flight ones, frees the server. */
bz_status bz_server_destroy(bz_server *srv);

/* Test of the certified FP32 threshold (Sec. 1 threshold, Table 1 forms):
 * the largest ratio |t32 - t64| / E over all pixels, where t64 is the
 * canonical FP64 threshold and t32, E the FP32 threshold and certified error
 * bound the BZ_FP64 kernels evaluate, taken over every evaluation form they
 * use (the two variance roundings and, for Sauvola with 0 <= k <= 1, the
 * form m (1 - k + (k/R) s)).  A ratio below 1 shows, for that image and
 * window, that every pixel the FP32 filter decides is decided as the FP64
 * threshold decides it.  method: 0 Sauvola, 1 Niblack, 3..7 Wolf, Feng,
 * Rais, NICK, Phansalkar; params as for binarize_precision_report_ext
 * ({k, R, ...}; Sauvola and Niblack read params[0] = k, params[1] = R).
 * max_ratio_dev: one device double, which the call raises to the ratio with
 * an atomic maximum (initialise it to 0).  Asynchronous on `stream`. */
bz_status binarize_bound_report(int32_t method, const uint8_t *image, int64_t H,
                                int64_t W, int64_t in_pitch, int32_t h,
                                int32_t w, const double *params,
                                double *max_ratio_dev, void *stream);

/* Debug build (libbinarize_debug.so, compiled with -DBZ_DEBUG; no
 * counterpart in the paper): every global load and store of the window,
 * small-page, stripe, quantile, min/max, Haar, batch and Table 1 kernels is
 * checked against the extent of its buffer; an access outside sets a status
 * bit (1 image load, 2 output store, 4 library scratch), records the first
 * offending address and is skipped, without trapping.  bz_debug_status
 * synchronizes with the device, returns the accumulated bits and address
 * (clearing them when reset != 0) and returns 0; in the normal build it
 * returns 1 with status 0.  -1 on a NULL argument or a CUDA error. */
int32_t bz_debug_status(uint32_t *status, uint64_t *first_addr, int32_t reset);

/* ---------------------------------------------------------------------- */
/* Autotuning of launch parameters (no counterpart in the paper: how the  */
/* work of Algorithm 1 and Sec. 3.4 is split over the GPU).               */
/* ---------------------------------------------------------------------- */
/* Tuned: the window kernel's tile height, edge-tile fraction and stripe
 * pre-pass (Sauvola / Niblack in every binarize precision), the quantile
 * kernel's row-band height, and the batched kernels' tile rows (multiples of
 * each job's window height).  Every candidate computes the same bits; only
 * the work split and so the time changes.  Candidates are timed with CUDA
 * events on the call's stream and the fastest is kept in a JSON cache keyed
 * by GPU name and SM count, kernel, precision (or quantile class: q < 1/4,
 * 1/4 <= q <= 3/4, q > 3/4), window buckets (next power of two of h and of w)
 * and image-size bucket (floor(2 log2(H W))).
 *   Environment: BZ_TUNE unset - launches use cached entries and never tune
 *   by themselves; BZ_TUNE=0 - the cache is ignored (built-in heuristics);
 *   BZ_TUNE=1 - a launch without a cached entry tunes itself first
 *   (synchronously).  BZ_TILE_ROWS, BZ_EDGE_FRAC and BZ_STRIPES, when set,
 *   take precedence over the cache.  The cache file is BZ_TUNE_CACHE, else
 *   $XDG_CACHE_HOME/paper_1905_13038_gb300/tune.json, else
 *   $HOME/.cache/paper_1905_13038_gb300/tune.json; a missing or malformed
 *   file reads as an empty cache and is rewritten whole after each tuning. */

/* Explicit tuning: performs the same binarization as binarize_sauvola
 * (method 0) / binarize_niblack (method 1) / binarize_quantile /
 * binarize_batch with the same arguments and errors, tuning first (the call
 * synchronizes `stream`), stores the winner and returns it: tile_h (0 when
 * the call takes a path without tunable parameters, the small-page kernel),
 * edge fraction (1 = uniform tiles), stripes (0/1), us = measured
 * microseconds per call; the batch returns its window and quantile tile
 * multipliers.  Each output pointer may be NULL. */
bz_status bz_autotune_window(int32_t method, const uint8_t *image, int64_t H,
                             int64_t W, int64_t in_pitch, int32_t h, int32_t w,
                             double k, double R, uint8_t *out, int64_t out_pitch,
                             bz_precision precision, void *stream,
                             int32_t *tile_h, float *edge, int32_t *stripes,
                             float *us);
bz_status bz_autotune_quantile(const uint8_t *image, int64_t H, int64_t W,
                               int64_t in_pitch, int32_t h, int32_t w,
                               int32_t q_num, int32_t q_den, int32_t offset,
                               uint8_t *out, int64_t out_pitch, void *stream,
                               int32_t *tile_h, float *us);
bz_status bz_autotune_batch(const bz_job *jobs_host, int32_t n,
                            bz_precision precision, void *stream,
                            int32_t *win_mult, int32_t *quant_mult, float *us);

/* Cache access (host only, no GPU needed).  Keys are built by bz_tune_key
 * from a GPU tag ("<name>/<SMs>"), a kernel ("window", "quantile",
 * "batch"), a class (window: 0 BZ_FP64, 1 BZ_FP32, 2 BZ_FP64_DIRECT;
 * quantile: the q class above; batch: the precision), h, w, H, W; it writes
 * the NUL-terminated key to buf (len bytes) and returns its length, or -1.
 * bz_tune_get: 1 and the fields when the key is cached, 0 when not, -1 on a
 * NULL key.  bz_tune_set: stores an entry in memory (0, or -1 on a bad
 * field: tile_h < 0, edge outside [0, 1], stripes outside [-1, 64]).
 * bz_tune_load: replaces the in-memory cache by the file's (path NULL: the
 * default path) and returns the number of entries, -1 when the file cannot
 * be read, -2 when it is malformed (the cache is then empty).  bz_tune_save:
 * writes the cache (path NULL: the path last loaded), 0 or -1.
 * bz_tune_window_plan: the window-kernel plan a binarize launch of an
 * H x W image would use on a GPU tagged `gpu` with `sms` SMs, cache
 * included: out[0..5] = tile_h, edge_h, edge tiles, tiles, stripes, resident
 * warps; returns 1 when a cached entry applied, 0 for the heuristics, -1 on
 * bad arguments. */
int32_t bz_tune_key(const char *gpu, const char *kernel, int32_t cls, int32_t h,
                    int32_t w, int64_t H, int64_t W, char *buf, int32_t len);
int32_t bz_tune_get(const char *key, int32_t *tile_h, float *edge,
                    int32_t *stripes, float *us);
int32_t bz_tune_set(const char *key, int32_t tile_h, float edge,
                    int32_t stripes, float us);
int32_t bz_tune_load(const char *path);
int32_t bz_tune_save(const char *path);
void bz_tune_clear(void);
int32_t bz_tune_window_plan(const char *gpu, int32_t precision, int64_t H,
                            int64_t W, int32_t h, int32_t w, int32_t sms,
                            int64_t *out);

#ifdef __cplusplus
}
#endif

#endif /* BINARIZE_H */
