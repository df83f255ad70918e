// Window-statistics kernels: Sauvola / Niblack binarization (FP64-exact,
// FP32, FP64-direct), the exact window-sum export and the FP32-vs-FP64
// report.  The per-tile arithmetic lives in bz_window.cuh.
#include <math.h>
#include <stdlib.h>

#include "bz_internal.h"

namespace bz {


// AW > 0: every tile takes the pipelined path with AW anchor words per lane
// (the host checked pipe_words); the variants are separate kernels so that
// each gets its own register allocation.  `stripes` (uniform schedules only):
// column sums at the first row of every tile row.
template <int MODE, bool VEC, typename S2T, bool WARMB, int AW>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kBlocksPerSM)
    k_window(Image g, Window win, Thresh T, Outputs o, TileSched S, const uint2 *stripes)
{
    __shared__ uint4 slots[kWarpsPerBlock][AW ? kPipeSlots : 1];  // pipelined path
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock;
    auto tile_of = [&](int64_t t, int64_t &tx, int64_t &y0, int64_t &y1, const uint2 *&st) {
        sched_tile(S, g.W, stripes, t, tx, y0, y1, st);
    };
    // let the next kernel be scheduled; prefetch this warp's first tile
    // into L2 while the previous kernel drains (a prefetch reads no result of
    // it), then wait for that kernel
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (S.prefetch && wid < S.tiles_total) {
        int64_t tx, y0, y1;
        const uint2 *st;
        tile_of(wid, tx, y0, y1, st);
        tile_prefetch_l2(g, win, tx * kTileCols, y0, y1, lane);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    fallbacks_clear(o);
    for (int64_t t = wid; t < S.tiles_total; t += stride) {
        int64_t tx, y0, y1;
        const uint2 *st;
        tile_of(t, tx, y0, y1, st);
        window_tile<MODE, VEC, S2T, AW, WARMB>(g, win, T, o, tx * kTileCols, y0, y1, lane,
                                                  slots[threadIdx.x >> 5], st, S.prefetch != 0 && t != wid);
    }
}

// Relative error bound of the FP32 evaluation in decide_f32 (units of
// 2^-24): inputs rounded once each, 1/n from two correctly rounded
// reciprocals and a product, sqrt.approx within 2^-22, one fused
// multiply-add per term and the rounding of the comparison operands; the
// derivation sums to < 18 units, 24 leaves a margin.
constexpr float kEpsF32 = 24.0f / 16777216.0f;

Thresh make_thresh(int method, double k, double R)
{
    Thresh T{};
    T.method = method;
    T.k = k;
    T.R = R;
    double alpha, beta, gamma, mag;
    const double u64 = 1.1102230246251565e-16;  // 2^-53
    if (method == 0) {  // Sauvola: t = m(1-k) + (k/R) m s
        alpha = 1.0 - k;
        beta = k / R;
        gamma = 0.0;
        // |t64 - t| <= 8 u64 m (1 + |k|(s/R + 1)), m <= 255, s <= 127.5
        mag = 16.0 * u64 * 255.0 * (1.0 + fabs(k) * (127.5 / R + 1.0));
    } else {  // Niblack: t = m + k s
        alpha = 1.0;
        beta = 0.0;
        gamma = k;
        mag = 8.0 * u64 * (255.0 + fabs(k) * 127.5);
    }
    T.alpha = (float)alpha;
    T.beta = (float)beta;
    T.gamma = (float)gamma;
    T.aalpha = fabsf(T.alpha);
    T.abeta = fabsf(T.beta);
    T.agamma = fabsf(T.gamma);
    T.eps = kEpsF32;
    T.delta64 = (float)(mag * 1.01) + 1e-30f;
    // Interior pipelined form (row constants alpha/n, gamma/n, beta/n^2 from
    // 1/n with 3 roundings; V and S1 rounded once; sqrt.approx within
    // 2^-22; three fused operations): |d32 - (t - I)| <= 17 u (M + 255),
    // u = 2^-24, M = |alpha| 255 + (|beta| 255 + |gamma|) 127.5 the largest
    // magnitude of the terms of t.  32 u (M + 256) leaves a margin.
    const double M = fabs(alpha) * 255.0 + (fabs(beta) * 255.0 + fabs(gamma)) * 127.5;
    T.bnd_c = (float)(32.0 / 16777216.0 * (M + 256.0)) + T.delta64;
    return T;
}

// Column band (ntx > 0): only the tile columns [tx0, tx0 + ntx) of rows
// [row0, row1), on a uniform one-wave schedule of their own and without the
// stripe pre-pass (it would cover every column).
struct ColBand {
    int64_t tx0 = 0, ntx = 0;
};

template <int MODE, bool VEC, typename S2T, bool WARMB>
static cudaError_t launch_t(const Image &g, const Window &win, const Thresh &T, const Outputs &o,
                            int64_t row0, int64_t row1, const ColBand &cb, cudaStream_t stream)
{
    constexpr bool kCanPipe = VEC && (MODE == MODE_FP64 || MODE == MODE_FP32) && sizeof(S2T) == 4;
    const int aw = kCanPipe ? pipe_words(MODE, VEC, sizeof(S2T) == 4, g, win) : 0;
    const bool pipe = aw > 0;
    uint2 *stripes = nullptr;
    TileSched S;
    if (cb.ntx > 0) {
        S.tiles_x = cb.ntx;
        S.tile_h = one_wave_tile_rows(row1 - row0, cb.ntx * kTileCols);
        S.edge_h = S.tile_h;
        S.n_edge = 0;
        S.row0 = row0;
        S.row1 = row1;
        S.tx0 = cb.tx0;
        S.tiles_total = cb.ntx * ((row1 - row0 + S.tile_h - 1) / S.tile_h);
        S.prefetch = 1;
    } else {
        const int64_t tile_h0 = window_tile_rows(row1 - row0, g.W, win.h, win.w);
        const int64_t tiles_y0 = (row1 - row0 + tile_h0 - 1) / tile_h0;
        stripes = launch_stripes(g, win, row0, tile_h0, tiles_y0, stream);
        S = make_sched(g, win, row0, row1, pipe, stripes != nullptr);
    }
    int64_t blocks = (S.tiles_total + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks > 2147483647LL)
        blocks = 2147483647LL;
    const uint2 *cst = stripes;
    cudaError_t e;
    if (aw == 1)
        e = launch_pdl(k_window<MODE, VEC, S2T, WARMB, kCanPipe ? 1 : 0>, (unsigned)blocks, 32 * kWarpsPerBlock,
                       stream, g, win, T, o, S, cst);
    else if (aw == 2)
        e = launch_pdl(k_window<MODE, VEC, S2T, WARMB, kCanPipe ? 2 : 0>, (unsigned)blocks, 32 * kWarpsPerBlock,
                       stream, g, win, T, o, S, cst);
    else
        e = launch_pdl(k_window<MODE, VEC, S2T, WARMB, 0>, (unsigned)blocks, 32 * kWarpsPerBlock, stream, g, win,
                       T, o, S, cst);
    if (stripes && scratch_free(stripes, stream) != cudaSuccess && e == cudaSuccess)
        e = cudaGetLastError();
    return e;
}

template <int MODE>
static cudaError_t launch_m(const Image &g, const Window &win, const Thresh &T, const Outputs &o,
                            int64_t row0, int64_t row1, cudaStream_t stream, const ColBand &cb = ColBand())
{
    if (cb.ntx == 0 && small_path_applies(MODE, g, win, row0, row1))
        return launch_small(MODE, g, win, T, o, row0, row1, stream);
    const bool vec = ((uintptr_t)g.img % 8 == 0) && (g.pitch % 8 == 0);
    const bool wide = (int64_t)win.h * win.w > 66051;  // S2 may reach 2^32
    if (MODE == MODE_REPORT) {  // the FP32 form the report follows
        Outputs o2 = o;
        o2.report_path = small_path_applies(MODE_FP32, g, win, row0, row1) ? kReportSmall
                         : (vec && !wide && pipe_words(MODE_FP32, true, true, g, win) > 0) ? kReportPipe
                                                                                       : kReportGeneric;
        return vec ? (wide ? launch_t<MODE, true, unsigned long long, false>(g, win, T, o2, row0, row1, cb, stream)
                           : launch_t<MODE, true, uint32_t, false>(g, win, T, o2, row0, row1, cb, stream))
                   : (wide ? launch_t<MODE, false, unsigned long long, false>(g, win, T, o2, row0, row1, cb, stream)
                           : launch_t<MODE, false, uint32_t, false>(g, win, T, o2, row0, row1, cb, stream));
    }
    // short tiles (a small image): the launch is latency-bound, so the
    // warm-up issues its loads in batches (binarize modes only)
    static const int env_warmb = [] {  // BZ_WARMB=0/1 forces it (tuning)
        const char *e = getenv("BZ_WARMB");
        return e ? atoi(e) : -1;
    }();
    const bool warmb = (MODE == MODE_FP64 || MODE == MODE_FP32) &&
                       (env_warmb >= 0 ? env_warmb != 0
                                       : (cb.ntx > 0 ? one_wave_tile_rows(row1 - row0, cb.ntx * kTileCols)
                                                     : window_tile_rows(row1 - row0, g.W, win.h, win.w)) <= 4);
    constexpr bool kB = (MODE == MODE_FP64 || MODE == MODE_FP32);
    if (warmb) {
        if (vec)
            return wide ? launch_t<MODE, true, unsigned long long, kB>(g, win, T, o, row0, row1, cb, stream)
                        : launch_t<MODE, true, uint32_t, kB>(g, win, T, o, row0, row1, cb, stream);
        return wide ? launch_t<MODE, false, unsigned long long, kB>(g, win, T, o, row0, row1, cb, stream)
                    : launch_t<MODE, false, uint32_t, kB>(g, win, T, o, row0, row1, cb, stream);
    }
    if (vec)
        return wide ? launch_t<MODE, true, unsigned long long, false>(g, win, T, o, row0, row1, cb, stream)
                    : launch_t<MODE, true, uint32_t, false>(g, win, T, o, row0, row1, cb, stream);
    return wide ? launch_t<MODE, false, unsigned long long, false>(g, win, T, o, row0, row1, cb, stream)
                : launch_t<MODE, false, uint32_t, false>(g, win, T, o, row0, row1, cb, stream);
}

// Binarize launches on the window kernel read their tile height, edge-tile
// fraction and stripe choice from the autotuner's cache (tune.cu); the
// window-sum export and the precision report keep the heuristics.
static bool window_tunable(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1)
{
    return (mode == MODE_FP64 || mode == MODE_FP32 || mode == MODE_FP64_DIRECT) &&
           !small_path_applies(mode, g, win, row0, row1);
}

cudaError_t launch_window_rows(int mode, const Image &g, const Window &win, const Thresh &T,
                               const Outputs &o, int64_t row0, int64_t row1, cudaStream_t stream)
{
    if (row0 < 0 || row1 > g.H || row0 >= row1)
        return cudaErrorInvalidValue;
    auto run = [&]() -> cudaError_t {
        switch (mode) {
        case MODE_FP64: return launch_m<MODE_FP64>(g, win, T, o, row0, row1, stream);
        case MODE_FP32: return launch_m<MODE_FP32>(g, win, T, o, row0, row1, stream);
        case MODE_FP64_DIRECT: return launch_m<MODE_FP64_DIRECT>(g, win, T, o, row0, row1, stream);
        case MODE_SUMS: return launch_m<MODE_SUMS>(g, win, T, o, row0, row1, stream);
        case MODE_REPORT: return launch_m<MODE_REPORT>(g, win, T, o, row0, row1, stream);
        default: return cudaErrorInvalidValue;
        }
    };
    if (!window_tunable(mode, g, win, row0, row1) || (tune_env() == 0 && !tune_forced()))
        return run();
    const std::string key = window_tune_key(mode, win, row1 - row0, g.W);
    TuneCfg c;
    bool have = tune_get(key, c);
    if (tune_now(have)) {
        const bool vec = ((uintptr_t)g.img % 8 == 0) && (g.pitch % 8 == 0);
        const bool pipe = pipe_words(mode, vec, (int64_t)win.h * win.w <= 66051, g, win) > 0;
        TuneCfg b;
        if (tune_window(mode, g, win, row0, row1, pipe, run, stream, b)) {
            c = b;
            have = true;
            tune_put(key, c, true);
            // the timed runs added to the FP64-fallback counter: count this
            // call's own launch only
            if (o.fallbacks && cudaMemsetAsync(o.fallbacks, 0, sizeof(unsigned long long), stream) != cudaSuccess)
                return cudaGetLastError();
        }
    }
    TuneScope scope(have ? &c : nullptr);
    return run();
}

cudaError_t launch_window_cols(int mode, const Image &g, const Window &win, const Thresh &T,
                               const Outputs &o, int64_t col0, int64_t col1, cudaStream_t stream)
{
    if (col0 < 0 || col0 % kTileCols != 0 || col1 <= col0 || col1 > g.W)
        return cudaErrorInvalidValue;
    ColBand cb;
    cb.tx0 = col0 / kTileCols;
    cb.ntx = (col1 - col0 + kTileCols - 1) / kTileCols;
    switch (mode) {
    case MODE_FP64: return launch_m<MODE_FP64>(g, win, T, o, 0, g.H, stream, cb);
    case MODE_FP32: return launch_m<MODE_FP32>(g, win, T, o, 0, g.H, stream, cb);
    case MODE_FP64_DIRECT: return launch_m<MODE_FP64_DIRECT>(g, win, T, o, 0, g.H, stream, cb);
    default: return cudaErrorInvalidValue;
    }
}

int window_kernel_count(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1)
{
    if (small_path_applies(mode, g, win, row0, row1))
        return 1;
    TuneCfg c;
    const bool have = window_tunable(mode, g, win, row0, row1) && tune_env() != 0 &&
                      tune_get(window_tune_key(mode, win, row1 - row0, g.W), c);
    TuneScope scope(have ? &c : nullptr);
    const int64_t tile_h = window_tile_rows(row1 - row0, g.W, win.h, win.w);
    const int64_t tiles_y = (row1 - row0 + tile_h - 1) / tile_h;
    return 1 + stripe_kernel_count(win, tile_h, tiles_y);
}

cudaError_t launch_window(int mode, const Image &g, const Window &win, const Thresh &T,
                          const Outputs &o, cudaStream_t stream)
{
    return launch_window_rows(mode, g, win, T, o, 0, g.H, stream);
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_window)

}  // namespace bz
