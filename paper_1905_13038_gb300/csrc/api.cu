// C ABI entry points: argument validation, overlap checks, dispatch.
#include <math.h>
#include <stdlib.h>
#include <mutex>

#include "bz_internal.h"

namespace bz {

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

static size_t span_bytes(int64_t rows, int64_t pitch, int64_t last_row_bytes)
{
    return (size_t)((rows - 1) * pitch + last_row_bytes);
}

bz_status check_image(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                      int32_t w)
{
    if (!image || H < 1 || W < 1 || H > 2147483647LL || W > 2147483647LL || in_pitch < W)
        return BZ_EINVAL;
    if (h < 1 || w < 1 || h > 511 || w > 511)
        return BZ_EINVAL;
    // H * pitch must stay addressable
    if (in_pitch > (INT64_MAX / H))
        return BZ_EINVAL;
    return BZ_OK;
}

bz_status check_out(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                    const uint8_t *out, int64_t out_pitch)
{
    const int64_t wb = (W + 7) / 8;
    if (!out || out_pitch < wb || out_pitch > (INT64_MAX / H))
        return BZ_EINVAL;
    if (ranges_overlap(image, span_bytes(H, in_pitch, in_pitch), out, span_bytes(H, out_pitch, wb)))
        return BZ_EOVERLAP;
    return BZ_OK;
}

// Three 8-byte FP64-fallback counters per device (allocated zeroed on first
// use): slots 0 and 1 for single-image calls in turn, slot 2 for batches.
struct FbState {
    unsigned long long *c = nullptr;
    int tog = 0, last = 0;
};
static std::mutex g_fb_mu;
static FbState g_fb[64];

static unsigned long long *fb_counters(int device)
{
    if (device < 0 || device >= 64)
        return nullptr;
    if (!g_fb[device].c) {
        void *p = nullptr;
        if (cudaMalloc(&p, 3 * sizeof(unsigned long long)) != cudaSuccess)
            return nullptr;
        if (cudaMemset(p, 0, 3 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        g_fb[device].c = (unsigned long long *)p;
    }
    return g_fb[device].c;
}

FbSlot fallback_slot(int device)
{
    std::lock_guard<std::mutex> lk(g_fb_mu);
    FbSlot f;
    unsigned long long *c = fb_counters(device);
    if (!c)
        return f;
    FbState &st = g_fb[device];
    st.tog ^= 1;
    st.last = st.tog;
    f.use = c + st.tog;
    f.clear = c + (st.tog ^ 1);
    return f;
}

unsigned long long *fallback_counter(int device)
{
    std::lock_guard<std::mutex> lk(g_fb_mu);
    unsigned long long *c = fb_counters(device);
    return c ? c + 2 : nullptr;
}

void fallback_mark_batch(int device)
{
    std::lock_guard<std::mutex> lk(g_fb_mu);
    if (device >= 0 && device < 64)
        g_fb[device].last = 2;
}

bool finite_params(int method, double k, double R)
{
    if (!isfinite(k) || fabs(k) > 1e6)
        return false;
    if (method == 0 && (!isfinite(R) || R < 1e-6 || R > 1e9))
        return false;
    return true;
}

static bz_status run_threshold(int method, const uint8_t *image, int64_t H, int64_t W,
                               int64_t in_pitch, int32_t h, int32_t w, double k, double R,
                               uint8_t *out, int64_t out_pitch, bz_precision precision,
                               void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    st = check_out(image, H, W, in_pitch, out, out_pitch);
    if (st != BZ_OK)
        return st;
    if (!finite_params(method, k, R))
        return BZ_EINVAL;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = MODE_FP64; break;
    case BZ_FP32: mode = MODE_FP32; break;
    case BZ_FP64_DIRECT: mode = MODE_FP64_DIRECT; break;
    default: return BZ_EINVAL;
    }
    Image g{image, H, W, in_pitch};
    Window win = make_window(h, w);
    Thresh T = make_thresh(method, k, method == 0 ? R : 128.0);
    Outputs o{};
    o.bits = out;
    o.out_pitch = out_pitch;
    o.bits_bytes = dbg_extent(H, out_pitch, (W + 7) / 8);
    o.bits_bytes = dbg_extent(H, out_pitch, (W + 7) / 8);
    if (mode == MODE_FP64) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess)
            return BZ_ECUDA;
        const FbSlot fb = fallback_slot(dev);
        o.fallbacks = fb.use;
        o.fallbacks_clear = fb.clear;
    }
    return launch_window(mode, g, win, T, o, (cudaStream_t)stream) == cudaSuccess ? BZ_OK
                                                                                  : BZ_ECUDA;
}

// Parameter ranges of the other Table 1 methods; prm = {k, R, alpha1, k1,
// k2, gamma, p, q}.  Every parameter is finite with |x| <= 1e6; R (where
// used) in [1e-6, 1e9]; Feng's gamma in [0, 16]; Phansalkar's q >= 0.
static bool ext_params_ok(int method, const double *prm)
{
    for (int i = 0; i < 8; i++)
        if (!isfinite(prm[i]) || fabs(prm[i]) > 1e6)
            return false;
    const bool usesR = method == METHOD_WOLF || method == METHOD_FENG || method == METHOD_PHANSALKAR;
    if (usesR && (prm[1] < 1e-6 || prm[1] > 1e9))
        return false;
    if (method == METHOD_FENG && (prm[5] < 0.0 || prm[5] > 16.0))
        return false;
    if (method == METHOD_PHANSALKAR && prm[7] < 0.0)
        return false;
    return method >= METHOD_WOLF && method <= METHOD_PHANSALKAR;
}

// The global sums need sum < 2^53 and N*sumsq < 2^128: H*W <= 2^44.
static bool global_size_ok(int64_t H, int64_t W)
{
    return (double)H * (double)W <= 17592186044416.0;
}

// Global statistics, then the window kernel reading them, on `stream`.
// The 24-byte GStats scratch is a stream-ordered allocation, freed on the
// stream after the kernel, so concurrent calls on different streams do not
// share it.
static bz_status run_ext(int method, const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                         int32_t h, int32_t w, const double *prm, int mode, Outputs o,
                         void *stream)
{
    if (!ext_params_ok(method, prm) || !global_size_ok(H, W))
        return BZ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Image g{image, H, W, in_pitch};
    GStats *gs = nullptr;
    if (scratch_alloc((void **)&gs, sizeof(GStats), s) != cudaSuccess)
        return BZ_ENOMEM;
    bz_status st = BZ_OK;
    const unsigned long long N = (unsigned long long)H * (unsigned long long)W;
    ThreshExt T = make_thresh_ext(method, prm, gs, N);
    if (launch_global_stats(g, gs, s) != cudaSuccess ||
        launch_window_ext(mode, g, make_window(h, w), T, o, s) != cudaSuccess)
        st = BZ_ECUDA;
    if (scratch_free(gs, s) != cudaSuccess)
        st = BZ_ECUDA;
    return st;
}

static bz_status run_ext_binarize(int method, const uint8_t *image, int64_t H, int64_t W,
                                  int64_t in_pitch, int32_t h, int32_t w, const double *prm,
                                  uint8_t *out, int64_t out_pitch, bz_precision precision,
                                  void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    st = check_out(image, H, W, in_pitch, out, out_pitch);
    if (st != BZ_OK)
        return st;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = MODE_FP64; break;
    case BZ_FP32: mode = MODE_FP32; break;
    case BZ_FP64_DIRECT: mode = MODE_FP64_DIRECT; break;
    default: return BZ_EINVAL;
    }
    Outputs o{};
    o.bits = out;
    o.out_pitch = out_pitch;
    o.bits_bytes = dbg_extent(H, out_pitch, (W + 7) / 8);
    o.bits_bytes = dbg_extent(H, out_pitch, (W + 7) / 8);
    if (mode == MODE_FP64) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess)
            return BZ_ECUDA;
        const FbSlot fb = fallback_slot(dev);
        o.fallbacks = fb.use;
        o.fallbacks_clear = fb.clear;
    }
    return run_ext(method, image, H, W, in_pitch, h, w, prm, mode, o, stream);
}

}  // namespace bz

using namespace bz;

extern "C" {

const char *bz_status_string(bz_status s)
{
    switch (s) {
    case BZ_OK: return "ok";
    case BZ_EINVAL: return "invalid argument";
    case BZ_EOVERLAP: return "image and output overlap";
    case BZ_ENOMEM: return "out of memory";
    case BZ_EBUDGET: return "request exceeds the HBM budget";
    case BZ_ECUDA: return "CUDA error";
    case BZ_ETIMEOUT: return "timed out";
    case BZ_EDEVICE_TIMEOUT: return "device-side wait timed out";
    case BZ_ECANCELLED: return "cancelled";
    }
    return "unknown status";
}

bz_status binarize_sauvola(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                           int32_t h, int32_t w, double k, double R, uint8_t *out,
                           int64_t out_pitch, bz_precision precision, void *stream)
{
    return run_threshold(0, image, H, W, in_pitch, h, w, k, R, out, out_pitch, precision, stream);
}

bz_status binarize_niblack(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                           int32_t h, int32_t w, double k, uint8_t *out, int64_t out_pitch,
                           bz_precision precision, void *stream)
{
    return run_threshold(1, image, H, W, in_pitch, h, w, k, 128.0, out, out_pitch, precision,
                         stream);
}

bz_status binarize_quantile(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                            int32_t h, int32_t w, int32_t q_num, int32_t q_den, int32_t offset,
                            uint8_t *out, int64_t out_pitch, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    st = check_out(image, H, W, in_pitch, out, out_pitch);
    if (st != BZ_OK)
        return st;
    if (q_den < 1 || q_num < 0 || q_num > q_den || offset < -255 || offset > 255)
        return BZ_EINVAL;
    Image g{image, H, W, in_pitch};
    return launch_quantile(g, make_window(h, w), q_num, q_den, offset, out, out_pitch, nullptr,
                           (cudaStream_t)stream) == cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

bz_status window_sums(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                      int32_t w, uint32_t *S1, uint64_t *S2, uint32_t *n, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    const size_t img_bytes = (size_t)(H * in_pitch);
    const size_t HW = (size_t)(H * W);
    if ((S1 && ranges_overlap(image, img_bytes, S1, HW * 4)) ||
        (S2 && ranges_overlap(image, img_bytes, S2, HW * 8)) ||
        (n && ranges_overlap(image, img_bytes, n, HW * 4)))
        return BZ_EOVERLAP;
    Image g{image, H, W, in_pitch};
    Outputs o{};
    o.S1 = S1;
    o.S2 = S2;
    o.n = n;
    o.sums_n = H * W;
    Thresh T = make_thresh(0, 0.5, 128.0);
    return launch_window(MODE_SUMS, g, make_window(h, w), T, o, (cudaStream_t)stream) ==
                   cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

bz_status window_quantile(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                          int32_t w, int32_t q_num, int32_t q_den, uint8_t *Q, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    if (!Q || q_den < 1 || q_num < 0 || q_num > q_den)
        return BZ_EINVAL;
    if (ranges_overlap(image, (size_t)(H * in_pitch), Q, (size_t)(H * W)))
        return BZ_EOVERLAP;
    Image g{image, H, W, in_pitch};
    return launch_quantile(g, make_window(h, w), q_num, q_den, 0, nullptr, 0, Q,
                           (cudaStream_t)stream) == cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

bz_status binarize_precision_report(int32_t method, const uint8_t *image, int64_t H, int64_t W,
                                    int64_t in_pitch, int32_t h, int32_t w, double k, double R,
                                    uint64_t *flips_dev, double *max_abs_dt_dev, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    if ((method != 0 && method != 1) || !flips_dev || !max_abs_dt_dev)
        return BZ_EINVAL;
    if (!finite_params(method, k, R))
        return BZ_EINVAL;
    Image g{image, H, W, in_pitch};
    Outputs o{};
    o.flips = (unsigned long long *)flips_dev;
    o.maxdt_bits = (unsigned long long *)max_abs_dt_dev;
    Thresh T = make_thresh(method, k, method == 0 ? R : 128.0);
    return launch_window(MODE_REPORT, g, make_window(h, w), T, o, (cudaStream_t)stream) ==
                   cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

bz_status binarize_wolf(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                        int32_t w, double k, double R, uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream)
{
    const double prm[8] = {k, R, 0, 0, 0, 0, 0, 0};
    return run_ext_binarize(METHOD_WOLF, image, H, W, in_pitch, h, w, prm, out, out_pitch,
                            precision, stream);
}

bz_status binarize_feng(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                        int32_t w, double alpha1, double k1, double k2, double gamma, double R,
                        uint8_t *out, int64_t out_pitch, bz_precision precision, void *stream)
{
    const double prm[8] = {0, R, alpha1, k1, k2, gamma, 0, 0};
    return run_ext_binarize(METHOD_FENG, image, H, W, in_pitch, h, w, prm, out, out_pitch,
                            precision, stream);
}

bz_status binarize_rais(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                        int32_t w, double k, uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream)
{
    const double prm[8] = {k, 128.0, 0, 0, 0, 0, 0, 0};
    return run_ext_binarize(METHOD_RAIS, image, H, W, in_pitch, h, w, prm, out, out_pitch,
                            precision, stream);
}

bz_status binarize_nick(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                        int32_t w, double k, uint8_t *out, int64_t out_pitch,
                        bz_precision precision, void *stream)
{
    const double prm[8] = {k, 128.0, 0, 0, 0, 0, 0, 0};
    return run_ext_binarize(METHOD_NICK, image, H, W, in_pitch, h, w, prm, out, out_pitch,
                            precision, stream);
}

bz_status binarize_phansalkar(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                              int32_t h, int32_t w, double k, double R, double p, double q,
                              uint8_t *out, int64_t out_pitch, bz_precision precision,
                              void *stream)
{
    const double prm[8] = {k, R, 0, 0, 0, 0, p, q};
    return run_ext_binarize(METHOD_PHANSALKAR, image, H, W, in_pitch, h, w, prm, out, out_pitch,
                            precision, stream);
}

bz_status global_stats(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                       double *stats_dev, uint64_t *sums_dev, void *stream)
{
    if (!image || !stats_dev || H < 1 || W < 1 || H > 2147483647LL || W > 2147483647LL ||
        in_pitch < W || in_pitch > (INT64_MAX / H) || !global_size_ok(H, W))
        return BZ_EINVAL;
    const size_t img_bytes = (size_t)(H * in_pitch);
    if (ranges_overlap(image, img_bytes, stats_dev, 3 * sizeof(double)) ||
        (sums_dev && ranges_overlap(image, img_bytes, sums_dev, 3 * sizeof(uint64_t))))
        return BZ_EOVERLAP;
    cudaStream_t s = (cudaStream_t)stream;
    GStats *gs = nullptr;
    if (scratch_alloc((void **)&gs, sizeof(GStats), s) != cudaSuccess)
        return BZ_ENOMEM;
    Image g{image, H, W, in_pitch};
    bz_status st = BZ_OK;
    if (launch_global_stats(g, gs, s) != cudaSuccess ||
        launch_global_finalize(gs, (unsigned long long)H * (unsigned long long)W, stats_dev,
                               sums_dev, s) != cudaSuccess)
        st = BZ_ECUDA;
    if (scratch_free(gs, s) != cudaSuccess)
        st = BZ_ECUDA;
    return st;
}

bz_status binarize_precision_report_ext(int32_t method, const uint8_t *image, int64_t H,
                                        int64_t W, int64_t in_pitch, int32_t h, int32_t w,
                                        const double *params, uint64_t *flips_dev,
                                        double *max_abs_dt_dev, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    if (!params || !flips_dev || !max_abs_dt_dev)
        return BZ_EINVAL;
    if (method == METHOD_SAUVOLA || method == METHOD_NIBLACK)
        return binarize_precision_report(method, image, H, W, in_pitch, h, w, params[0],
                                         params[1], flips_dev, max_abs_dt_dev, stream);
    Outputs o{};
    o.flips = (unsigned long long *)flips_dev;
    o.maxdt_bits = (unsigned long long *)max_abs_dt_dev;
    return run_ext(method, image, H, W, in_pitch, h, w, params, MODE_REPORT, o, stream);
}

bz_status window_minmax(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                        int32_t w, uint8_t *mn, uint8_t *mx, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    if (!mn || !mx)
        return BZ_EINVAL;
    const size_t img_bytes = (size_t)(H * in_pitch);
    const size_t HW = (size_t)(H * W);
    if (ranges_overlap(image, img_bytes, mn, HW) || ranges_overlap(image, img_bytes, mx, HW) ||
        ranges_overlap(mn, HW, mx, HW))
        return BZ_EOVERLAP;
    Image g{image, H, W, in_pitch};
    return launch_minmax(g, make_window(h, w), 0, mn, mx, nullptr, 0, (cudaStream_t)stream) ==
                   cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

bz_status binarize_bernsen(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                           int32_t h, int32_t w, int32_t contrast_limit, uint8_t *out,
                           int64_t out_pitch, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    st = check_out(image, H, W, in_pitch, out, out_pitch);
    if (st != BZ_OK)
        return st;
    if (contrast_limit < 0 || contrast_limit > 256)
        return BZ_EINVAL;
    Image g{image, H, W, in_pitch};
    return launch_minmax(g, make_window(h, w), contrast_limit, nullptr, nullptr, out, out_pitch,
                         (cudaStream_t)stream) == cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

bz_status haar_feature(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                       const bz_haar *feature, int32_t *out, void *stream)
{
    if (!feature || !out)
        return BZ_EINVAL;
    const bz_haar &F = *feature;
    if (F.n_row < 1 || F.n_row > 4 || F.n_col < 1 || F.n_col > 4)
        return BZ_EINVAL;
    int32_t h = 0, w = 0, fmax = 0, gmax = 0;
    for (int s = 0; s < F.n_row; s++) {
        if (F.row_len[s] < 1 || F.row_len[s] > 511 || F.row_wt[s] < -127 || F.row_wt[s] > 127)
            return BZ_EINVAL;
        h += F.row_len[s];
        fmax = abs(F.row_wt[s]) > fmax ? abs(F.row_wt[s]) : fmax;
    }
    for (int s = 0; s < F.n_col; s++) {
        if (F.col_len[s] < 1 || F.col_len[s] > 511 || F.col_wt[s] < -127 || F.col_wt[s] > 127)
            return BZ_EINVAL;
        w += F.col_len[s];
        gmax = abs(F.col_wt[s]) > gmax ? abs(F.col_wt[s]) : gmax;
    }
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    // |feature| <= 255 h w max|f| max|g| must stay below 2^31
    if (255.0 * h * w * fmax * gmax > 2147483647.0)
        return BZ_EINVAL;
    const size_t img_bytes = (size_t)(H * in_pitch);
    if (ranges_overlap(image, img_bytes, out, (size_t)(H * W) * sizeof(int32_t)))
        return BZ_EOVERLAP;
    HaarDev hd{};
    hd.n_rs = F.n_row;
    for (int s = 0; s < F.n_row; s++) {
        hd.rs_len[s] = F.row_len[s];
        hd.rs_wt[s] = F.row_wt[s];
    }
    // taps at the segment boundaries: coefficient f(a-1) - f(a), f = 0 outside
    int a = 0;
    for (int s = 0; s <= F.n_row; s++) {
        const int before = s > 0 ? F.row_wt[s - 1] : 0, after = s < F.n_row ? F.row_wt[s] : 0;
        if (before != after) {
            hd.rt_a[hd.n_rt] = a;
            hd.rt_c[hd.n_rt] = before - after;
            hd.n_rt++;
        }
        if (s < F.n_row)
            a += F.row_len[s];
    }
    int b = 0;
    for (int s = 0; s <= F.n_col; s++) {
        const int before = s > 0 ? F.col_wt[s - 1] : 0, after = s < F.n_col ? F.col_wt[s] : 0;
        if (before != after) {
            hd.ct_b[hd.n_ct] = b;
            hd.ct_c[hd.n_ct] = before - after;
            hd.n_ct++;
        }
        if (s < F.n_col)
            b += F.col_len[s];
    }
    Image g{image, H, W, in_pitch};
    return launch_haar(g, make_window(h, w), hd, out, (cudaStream_t)stream) == cudaSuccess
               ? BZ_OK
               : BZ_ECUDA;
}

// Column bands (Sec. 3.3's exchanged axes applied to the in-place mode):
// band k covers the output columns [c0, c1) of every row, c0 = k B.  Its
// packed bits are written to a scratch of H rows x B/8 bytes and then copied
// to bytes [c0/8, ceil(c1/8)) of each image row at once: later bands read
// only columns >= c1 - l + 1 (their windows start there), and with
// 7 c1 / 8 >= l - 1 every overwritten column c < c1 / 8 lies left of that.
// The first band ends at c1 = B, so B = 256 serves l <= 225 and B = 512
// every window up to 511; later bands end further right.  One scratch slot
// suffices: the copy of band k is ordered after band k on the stream and
// before band k + 1.
static int64_t inplace_band_cols(int32_t w, int64_t band_cols)
{
    const int64_t l = (w + 1) / 2;
    const int64_t bmin = (l - 1) * 8 <= 7 * 256 ? 256 : 512;
    if (band_cols == 0)
        return bmin;
    if (band_cols < bmin || band_cols % 256 != 0)
        return -1;
    return band_cols;
}

bz_status binarize_inplace(int32_t method, uint8_t *image, int64_t H, int64_t W, int64_t pitch,
                           int32_t h, int32_t w, double k, double R, int64_t band_rows,
                           bz_precision precision, void *stream)
{
    bz_status st = check_image(image, H, W, pitch, h, w);
    if (st != BZ_OK)
        return st;
    if ((method != 0 && method != 1) || !finite_params(method, k, R))
        return BZ_EINVAL;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = MODE_FP64; break;
    case BZ_FP32: mode = MODE_FP32; break;
    case BZ_FP64_DIRECT: mode = MODE_FP64_DIRECT; break;
    default: return BZ_EINVAL;
    }
    const Window win = make_window(h, w);
    const int64_t B = band_rows == 0 ? (win.o > 256 ? win.o : 256) : band_rows;
    if (B < win.o)
        return BZ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t cw = (W + 7) / 8;
    Image g{image, H, W, pitch};
    Thresh T = make_thresh(method, k, method == 0 ? R : 128.0);
    unsigned long long *fb = nullptr, *fbc = nullptr;
    if (mode == MODE_FP64) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess)
            return BZ_ECUDA;
        const FbSlot f = fallback_slot(dev);
        fb = f.use;
        fbc = f.clear;
    }
    const int64_t band = B < H ? B : H;
    uint8_t *scratch = nullptr;
    if (scratch_alloc((void **)&scratch, (size_t)(2 * band * cw), s) != cudaSuccess)
        return BZ_ENOMEM;
    // Band k is binarized into scratch slot k % 2 while the image still holds
    // every gray level its windows need; band k-1 is copied into place only
    // after band k has run.  Band k+1 reads rows >= start(k+1) - o + 1, which
    // lie in band k or later because B >= o, so it never sees an overwritten
    // row.
    int64_t prev_row0 = -1, prev_rows = 0;
    int slot = 0;
    for (int64_t r0 = 0; r0 < H && st == BZ_OK; r0 += band, slot ^= 1) {
        const int64_t r1 = r0 + band < H ? r0 + band : H;
        Outputs o{};
        o.bits = scratch + (int64_t)slot * band * cw;
        o.out_pitch = cw;
        o.out_row0 = r0;
        o.bits_bytes = (size_t)band * cw;
        o.fallbacks = fb;
        o.fallbacks_clear = fbc;
        if (launch_window_rows(mode, g, win, T, o, r0, r1, s) != cudaSuccess)
            st = BZ_ECUDA;
        else if (prev_row0 >= 0 &&
                 cudaMemcpy2DAsync(image + prev_row0 * pitch, (size_t)pitch,
                                   scratch + (int64_t)(slot ^ 1) * band * cw, (size_t)cw,
                                   (size_t)cw, (size_t)prev_rows, cudaMemcpyDeviceToDevice,
                                   s) != cudaSuccess)
            st = BZ_ECUDA;
        prev_row0 = r0;
        prev_rows = r1 - r0;
    }
    if (st == BZ_OK &&
        cudaMemcpy2DAsync(image + prev_row0 * pitch, (size_t)pitch,
                          scratch + (int64_t)(slot ^ 1) * band * cw, (size_t)cw, (size_t)cw,
                          (size_t)prev_rows, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = BZ_ECUDA;
    if (scratch_free(scratch, s) != cudaSuccess)
        st = BZ_ECUDA;
    return st;
}

bz_status binarize_inplace_cols(int32_t method, uint8_t *image, int64_t H, int64_t W, int64_t pitch,
                                int32_t h, int32_t w, double k, double R, int64_t band_cols,
                                bz_precision precision, void *stream)
{
    bz_status st = check_image(image, H, W, pitch, h, w);
    if (st != BZ_OK)
        return st;
    if ((method != 0 && method != 1) || !finite_params(method, k, R))
        return BZ_EINVAL;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = MODE_FP64; break;
    case BZ_FP32: mode = MODE_FP32; break;
    case BZ_FP64_DIRECT: mode = MODE_FP64_DIRECT; break;
    default: return BZ_EINVAL;
    }
    const int64_t B = inplace_band_cols(w, band_cols);
    if (B < 0)
        return BZ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Window win = make_window(h, w);
    const Image g{image, H, W, pitch};
    const Thresh T = make_thresh(method, k, method == 0 ? R : 128.0);
    unsigned long long *fb = nullptr, *fbc = nullptr;
    if (mode == MODE_FP64) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess)
            return BZ_ECUDA;
        const FbSlot f = fallback_slot(dev);
        fb = f.use;
        fbc = f.clear;
    }
    const int64_t slot_bytes = (B < W ? B : W + 7) / 8;  // bytes of a band's output row
    uint8_t *scratch = nullptr;
    if (scratch_alloc((void **)&scratch, (size_t)(H * slot_bytes), s) != cudaSuccess)
        return BZ_ENOMEM;
    for (int64_t c0 = 0; c0 < W && st == BZ_OK; c0 += B) {
        const int64_t c1 = c0 + B < W ? c0 + B : W;
        Outputs o{};
        o.bits = scratch;
        o.out_pitch = slot_bytes;
        o.out_byte0 = c0 / 8;
        o.bits_bytes = (size_t)(H * slot_bytes);
        o.fallbacks = fb;
        o.fallbacks_clear = fbc;
        const int64_t nbytes = (c1 + 7) / 8 - c0 / 8;
        if (launch_window_cols(mode, g, win, T, o, c0, c1, s) != cudaSuccess ||
            cudaMemcpy2DAsync(image + c0 / 8, (size_t)pitch, scratch, (size_t)slot_bytes, (size_t)nbytes,
                              (size_t)H, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            st = BZ_ECUDA;
    }
    if (scratch_free(scratch, s) != cudaSuccess)
        st = BZ_ECUDA;
    return st;
}

// binarize_host's per-device pipeline: an upload, a compute and a download
// stream, and two slots used in turn, each with a device image and output
// buffer and the events that mark its upload, compute and download done.
// Call n uploads into slot n % 2 once that slot's previous compute has read
// it, computes once the upload is done and the slot's previous output is
// home, and downloads each window's output as soon as that window's launch
// is done (one event per window, so a call's downloads run during its later
// windows' compute and only the last one is left after it); the caller's
// stream waits only for the downloads, so call n+1's upload runs during call
// n's compute and call n+1's compute during call n's last download.  Fixed
// buffers rather than stream-ordered
// allocations: a pool allocation on one stream can be handed memory freed on
// another and then wait for that stream's work.
struct HostSlot {
    uint8_t *img = nullptr, *out = nullptr;
    size_t img_cap = 0, out_cap = 0;
    cudaEvent_t up = nullptr, comp = nullptr, down = nullptr;
    cudaEvent_t win[64] = {};  // window q's launches done (created on first use)
};

struct HostState {
    std::mutex mu;
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    HostSlot slot[2];
    int next = 0;
};

static HostState *host_state(int dev)
{
    static std::mutex mu;
    static HostState *st[64] = {nullptr};
    if (dev < 0 || dev >= 64)
        return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!st[dev]) {
        HostState *h = new HostState();
        bool ok = cudaStreamCreateWithFlags(&h->up, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->comp, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->down, cudaStreamNonBlocking) == cudaSuccess;
        for (HostSlot &sl : h->slot)
            ok = ok && cudaEventCreateWithFlags(&sl.up, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.comp, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.down, cudaEventDisableTiming) == cudaSuccess;
        if (!ok)
            return nullptr;  // (leaked on this rare failure; the next call retries)
        st[dev] = h;
    }
    return st[dev];
}

// Grow a slot buffer to `need` bytes once its last user (marked by `last`)
// is done.
static bool host_grow(uint8_t *&buf, size_t &cap, size_t need, cudaEvent_t last)
{
    if (cap >= need)
        return true;
    if (cudaEventSynchronize(last) != cudaSuccess)
        return false;
    if (buf)
        cudaFree(buf);
    buf = nullptr;
    cap = 0;
    if (cudaMalloc((void **)&buf, need) != cudaSuccess)
        return false;
    cap = need;
    return true;
}

// One host-memory call over n windows of the same image: one upload, n
// window launches, n downloads (binarize_host is n = 1).
static bz_status host_run(int32_t method, const uint8_t *image_host, int64_t H, int64_t W, int64_t in_pitch,
                          int32_t n, const int32_t *hv, const int32_t *wv, double k, double R,
                          uint8_t *const *outs, int64_t out_pitch, bz_precision precision, void *stream)
{
    if (n < 1 || n > 64 || !hv || !wv || !outs)
        return BZ_EINVAL;
    for (int q = 0; q < n; q++) {
        const bz_status st = check_image(image_host, H, W, in_pitch, hv[q], wv[q]);
        if (st != BZ_OK)
            return st;
    }
    const int64_t cw = (W + 7) / 8;
    if (out_pitch < cw || out_pitch > (INT64_MAX / H))
        return BZ_EINVAL;
    const size_t in_span = (size_t)((H - 1) * in_pitch + W), out_span = (size_t)((H - 1) * out_pitch + cw);
    for (int q = 0; q < n; q++) {
        if (!outs[q])
            return BZ_EINVAL;
        if (ranges_overlap(image_host, in_span, outs[q], out_span))
            return BZ_EOVERLAP;
        for (int q2 = 0; q2 < q; q2++)
            if (ranges_overlap(outs[q2], out_span, outs[q], out_span))
                return BZ_EOVERLAP;
    }
    if ((method != 0 && method != 1) || !finite_params(method, k, R))
        return BZ_EINVAL;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = MODE_FP64; break;
    case BZ_FP32: mode = MODE_FP32; break;
    case BZ_FP64_DIRECT: mode = MODE_FP64_DIRECT; break;
    default: return BZ_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return BZ_ECUDA;
    HostState *hs = host_state(dev);
    if (!hs)
        return BZ_ECUDA;
    const Thresh T = make_thresh(method, k, method == 0 ? R : 128.0);
    // device rows of 16-byte multiples; a host pitch that already is one (and
    // no wider than needed) keeps the copy a single contiguous transfer
    const int64_t dpitch = (in_pitch % 16 == 0 && in_pitch - W < 16) ? in_pitch : (W + 15) & ~(int64_t)15;
    const size_t plane = (size_t)(H * cw);
    const FbSlot fbs = mode == MODE_FP64 ? fallback_slot(dev) : FbSlot();
    unsigned long long *fb = fbs.use;
    std::lock_guard<std::mutex> lk(hs->mu);
    HostSlot &sl = hs->slot[hs->next];
    hs->next ^= 1;
    bool ok = host_grow(sl.img, sl.img_cap, (size_t)(H * dpitch), sl.down) &&
              host_grow(sl.out, sl.out_cap, plane * (size_t)n, sl.down);
    // upload once the slot's previous compute has read its image
    ok = ok && cudaStreamWaitEvent(hs->up, sl.comp, 0) == cudaSuccess;
    if (ok && dpitch == in_pitch)
        ok = cudaMemcpyAsync(sl.img, image_host, in_span, cudaMemcpyHostToDevice, hs->up) == cudaSuccess;
    else if (ok)
        ok = cudaMemcpy2DAsync(sl.img, (size_t)dpitch, image_host, (size_t)in_pitch, (size_t)W, (size_t)H,
                               cudaMemcpyHostToDevice, hs->up) == cudaSuccess;
    ok = ok && cudaEventRecord(sl.up, hs->up) == cudaSuccess;
    // compute once the upload is done and the slot's previous outputs are home
    ok = ok && cudaStreamWaitEvent(hs->comp, sl.up, 0) == cudaSuccess &&
         cudaStreamWaitEvent(hs->comp, sl.down, 0) == cudaSuccess;
    for (int q = 0; ok && q < n; q++) {
        Outputs o{};
        o.bits = sl.out + plane * (size_t)q;
        o.out_pitch = cw;
        o.bits_bytes = plane;
        o.fallbacks = fb;
        o.fallbacks_clear = fbs.clear;
        ok = launch_window(mode, Image{sl.img, H, W, dpitch}, make_window(hv[q], wv[q]), T, o, hs->comp) ==
             cudaSuccess;
        if (ok && q + 1 < n) {  // window q's output can go home while the next ones compute
            if (!sl.win[q])
                ok = cudaEventCreateWithFlags(&sl.win[q], cudaEventDisableTiming) == cudaSuccess;
            ok = ok && cudaEventRecord(sl.win[q], hs->comp) == cudaSuccess;
        }
    }
    ok = ok && cudaEventRecord(sl.comp, hs->comp) == cudaSuccess;
    // downloads, each after its window's launches, and order the caller's
    // stream after them
    for (int q = 0; ok && q < n; q++) {
        ok = cudaStreamWaitEvent(hs->down, q + 1 < n ? sl.win[q] : sl.comp, 0) == cudaSuccess;
        if (!ok)
            break;
        const uint8_t *src = sl.out + plane * (size_t)q;
        if (out_pitch == cw)
            ok = cudaMemcpyAsync(outs[q], src, plane, cudaMemcpyDeviceToHost, hs->down) == cudaSuccess;
        else
            ok = cudaMemcpy2DAsync(outs[q], (size_t)out_pitch, src, (size_t)cw, (size_t)cw, (size_t)H,
                                   cudaMemcpyDeviceToHost, hs->down) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(sl.down, hs->down) == cudaSuccess &&
         cudaStreamWaitEvent((cudaStream_t)stream, sl.down, 0) == cudaSuccess;
    if (!ok) {  // leave nothing of this call in flight
        cudaStreamSynchronize(hs->up);
        cudaStreamSynchronize(hs->comp);
        cudaStreamSynchronize(hs->down);
    }
    return ok ? BZ_OK : BZ_ECUDA;
}

bz_status binarize_host(int32_t method, const uint8_t *image_host, int64_t H, int64_t W,
                        int64_t in_pitch, int32_t h, int32_t w, double k, double R,
                        uint8_t *out_host, int64_t out_pitch, bz_precision precision, void *stream)
{
    if (!out_host)
        return BZ_EINVAL;
    uint8_t *outs[1] = {out_host};
    return host_run(method, image_host, H, W, in_pitch, 1, &h, &w, k, R, outs, out_pitch, precision, stream);
}

bz_status binarize_host_multi(int32_t method, const uint8_t *image_host, int64_t H, int64_t W,
                              int64_t in_pitch, int32_t n, const int32_t *h, const int32_t *w, double k,
                              double R, uint8_t *const *out_host, int64_t out_pitch, bz_precision precision,
                              void *stream)
{
    return host_run(method, image_host, H, W, in_pitch, n, h, w, k, R, out_host, out_pitch, precision,
                    stream);
}

int64_t bz_inplace_cols_scratch_bytes(int64_t H, int64_t W, int32_t w, int64_t band_cols)
{
    if (H < 1 || W < 1 || w < 1 || w > 511)
        return -1;
    const int64_t B = inplace_band_cols(w, band_cols);
    if (B < 0)
        return -1;
    return H * ((B < W ? B : W + 7) / 8);
}

int64_t bz_inplace_scratch_bytes(int64_t H, int64_t W, int32_t h, int64_t band_rows)
{
    if (H < 1 || W < 1 || h < 1 || h > 511)
        return -1;
    const int64_t o = (h + 1) / 2;
    const int64_t B = band_rows == 0 ? (o > 256 ? o : 256) : band_rows;
    if (B < o)
        return -1;
    const int64_t band = B < H ? B : H;
    return 2 * band * ((W + 7) / 8);
}

bz_status binarize_bound_report(int32_t method, const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                                int32_t h, int32_t w, const double *params, double *max_ratio_dev, void *stream)
{
    bz_status st = check_image(image, H, W, in_pitch, h, w);
    if (st != BZ_OK)
        return st;
    if (!params || !max_ratio_dev)
        return BZ_EINVAL;
    Outputs o{};
    o.maxratio_bits = (unsigned long long *)max_ratio_dev;
    if (method == METHOD_SAUVOLA || method == METHOD_NIBLACK) {
        const double k = params[0], R = method == METHOD_SAUVOLA ? params[1] : 128.0;
        if (!finite_params(method, k, R))
            return BZ_EINVAL;
        const Thresh T = make_thresh(method, k, R);
        return launch_window(MODE_REPORT, Image{image, H, W, in_pitch}, make_window(h, w), T, o,
                             (cudaStream_t)stream) == cudaSuccess
                   ? BZ_OK
                   : BZ_ECUDA;
    }
    if (method < METHOD_WOLF || method > METHOD_PHANSALKAR)
        return BZ_EINVAL;
    return run_ext(method, image, H, W, in_pitch, h, w, params, MODE_REPORT, o, stream);
}

// ---- explicit tuning calls: the same work as the binarize call, with the
// autotuner's timed search forced for it (tune.cu); the chosen configuration
// is stored in the cache and returned.
bz_status bz_autotune_window(int32_t method, const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                             int32_t h, int32_t w, double k, double R, uint8_t *out, int64_t out_pitch,
                             bz_precision precision, void *stream, int32_t *tile_h, float *edge,
                             int32_t *stripes, float *us)
{
    if (method != 0 && method != 1)
        return BZ_EINVAL;
    bz_status st;
    {
        TuneForce force;
        st = run_threshold(method, image, H, W, in_pitch, h, w, k, method == 0 ? R : 128.0, out, out_pitch,
                           precision, stream);
    }
    if (st != BZ_OK)
        return st;
    const int mode = precision == BZ_FP64 ? MODE_FP64 : (precision == BZ_FP32 ? MODE_FP32 : MODE_FP64_DIRECT);
    TuneCfg c;  // zeros: the call took a path without tunable parameters
    tune_get(window_tune_key(mode, make_window(h, w), H, W), c);
    if (tile_h)
        *tile_h = c.tile_h;
    if (edge)
        *edge = c.edge;
    if (stripes)
        *stripes = c.stripes;
    if (us)
        *us = c.us;
    return BZ_OK;
}

bz_status bz_autotune_quantile(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                               int32_t w, int32_t q_num, int32_t q_den, int32_t offset, uint8_t *out,
                               int64_t out_pitch, void *stream, int32_t *tile_h, float *us)
{
    bz_status st;
    {
        TuneForce force;
        st = binarize_quantile(image, H, W, in_pitch, h, w, q_num, q_den, offset, out, out_pitch, stream);
    }
    if (st != BZ_OK)
        return st;
    TuneCfg c;
    tune_get(quantile_tune_key(q_num, q_den, make_window(h, w), H, W), c);
    if (tile_h)
        *tile_h = c.tile_h;
    if (us)
        *us = c.us;
    return BZ_OK;
}

bz_status bz_autotune_batch(const bz_job *jobs_host, int32_t n, bz_precision precision, void *stream,
                            int32_t *win_mult, int32_t *quant_mult, float *us)
{
    bz_status st;
    {
        TuneForce force;
        st = binarize_batch(jobs_host, n, precision, stream);
    }
    if (st != BZ_OK)
        return st;
    const int mode = precision == BZ_FP64 ? 0 : (precision == BZ_FP32 ? 1 : 2);
    TuneCfg c;
    tune_get(batch_tune_key(mode), c);
    if (win_mult)
        *win_mult = c.tile_h;
    if (quant_mult)
        *quant_mult = c.stripes;
    if (us)
        *us = c.us;
    return BZ_OK;
}

int32_t bz_kernels_per_call(int64_t H, int64_t W, int32_t h, int32_t w, bz_precision precision)
{
    if (H < 1 || W < 1 || h < 1 || w < 1)
        return -1;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = MODE_FP64; break;
    case BZ_FP32: mode = MODE_FP32; break;
    case BZ_FP64_DIRECT: mode = MODE_FP64_DIRECT; break;
    default: return -1;
    }
    const Image g{nullptr, H, W, (W + 7) & ~(int64_t)7};
    return window_kernel_count(mode, g, make_window(h, w), 0, H);
}

int32_t bz_tile_schedule(int64_t H, int64_t W, int32_t sms, int32_t pipe, int32_t stripes, int64_t *out)
{
    if (!out)
        return -1;
    return plan_tile_schedule(H, W, sms, pipe != 0, stripes != 0, out);
}

int32_t bz_debug_status(uint32_t *status, uint64_t *first_addr, int32_t reset)
{
    if (!status || !first_addr)
        return -1;
    unsigned st = 0;
    unsigned long long addr = 0;
    int r = 0;
    for (auto fn : {dbg_status_window, dbg_status_small, dbg_status_stripes, dbg_status_quantile, dbg_status_minmax,
                    dbg_status_haar, dbg_status_batch, dbg_status_table1}) {
        const int e = fn(&st, &addr, reset != 0);
        if (e < 0)
            return -1;
        r = e;  // 1 throughout in a normal build
    }
    *status = st;
    *first_addr = addr;
    return r;
}

int64_t bz_last_fp64_fallbacks(void *stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return -1;
    unsigned long long *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_fb_mu);
        if (dev >= 0 && dev < 64 && g_fb[dev].c)
            p = g_fb[dev].c + g_fb[dev].last;
    }
    if (!p)
        return 0;  // no BZ_FP64 call on this device yet
    unsigned long long v = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return -1;
    if (cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    return (int64_t)v;
}

}  // extern "C"
