// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>

#include "../../include/binarize.h"
#include "bz_window.cuh"

namespace bz {

// Window parameters of Algorithm 1.
// Launch `kernel` on `stream` with programmatic stream serialization, so that
// it may be scheduled while the previous kernel drains; the kernel must begin
// with pdl_begin().  BZ_PDL=0 launches plainly (tuning).
bool pdl_enabled();
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t stream,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

inline Window make_window(int h, int w)
{
    Window win;
    win.h = h;
    win.w = w;
    win.l = (w + 1) / 2;
    win.r = w / 2;
    win.o = (h + 1) / 2;
    win.u = h / 2;
    return win;
}

Thresh make_thresh(int method, double k, double R);

// Rows of a warp tile for the window path (autotuned heuristics).
int64_t window_tile_rows(int64_t H, int64_t W, int h, int w);

// Small pages, windows up to 63 x 63 (k_small.cu): shared-memory tiles
// instead of latency-bound warp tiles.
bool small_path_applies(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1);
cudaError_t launch_small(int mode, const Image &g, const Window &win, const Thresh &T,
                         const Outputs &o, int64_t row0, int64_t row1, cudaStream_t stream);

// Stripe pre-pass on `stream` for windows of at least 48 rows spanning five
// or more tile heights: (C, D) column
// sums at every tile start row0 + s * tile_h, s < tiles_y, in a stream-ordered
// scratch of tiles_y * W uint2 that the caller frees on the stream after the
// window kernel; nullptr when not used or not available.
uint2 *launch_stripes(const Image &g, const Window &win, int64_t row0, int64_t tile_h,
                      int64_t tiles_y, cudaStream_t stream);
// Kernels launch_stripes enqueues for this geometry (0: no stripes).
int stripe_kernel_count(const Window &win, int64_t tile_h, int64_t tiles_y);

// Window kernel geometry: 4 warps per block, 4 blocks per SM (128 registers
// per thread); one wave is SMs x 16 warps.
constexpr int kWarpsPerBlock = 4;
constexpr int kBlocksPerSM = 4;

// The tile schedule of a window-kernel launch over rows [row0, row1): one-wave
// interior tiles and, without stripes, shorter edge tiles (pipe: the edge
// tiles take the pipelined path, else the generic one).
TileSched make_sched(const Image &g, const Window &win, int64_t row0, int64_t row1, bool pipe, bool stripes);
// The same from H, W and an SM count alone (no device): tiles_x, tile_h,
// edge_h, n_edge, tiles_total and the resident warps into out[0..5].
int plan_tile_schedule(int64_t H, int64_t W, int sms, bool pipe, bool stripes, int64_t out[6]);

// Launches of the window path; mode is a bz::Mode.
cudaError_t launch_window(int mode, const Image &g, const Window &win, const Thresh &T,
                          const Outputs &o, cudaStream_t stream);
// Kernels one launch_window_rows call enqueues (stripe pre-pass included).
int window_kernel_count(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1);
// The same over the output rows [row0, row1) only (windows still see the
// whole image).
cudaError_t launch_window_rows(int mode, const Image &g, const Window &win, const Thresh &T,
                               const Outputs &o, int64_t row0, int64_t row1, cudaStream_t stream);
// Binarize modes over the output columns [col0, col1) of every row only
// (col0 a multiple of 256; windows still see the whole image); column j goes
// to output byte j / 8 - o.out_byte0.
cudaError_t launch_window_cols(int mode, const Image &g, const Window &win, const Thresh &T,
                               const Outputs &o, int64_t col0, int64_t col1, cudaStream_t stream);

// The other Table 1 methods (k_table1.cu).  prm = {k, R, alpha1, k1, k2,
// gamma, p, q}.
ThreshExt make_thresh_ext(int method, const double *prm, const GStats *gs, unsigned long long N);
cudaError_t launch_global_stats(const Image &g, GStats *gs, cudaStream_t stream);
cudaError_t launch_global_finalize(const GStats *gs, unsigned long long N, double *stats,
                                   uint64_t *sums, cudaStream_t stream);
cudaError_t launch_window_ext(int mode, const Image &g, const Window &win, const ThreshExt &T,
                              const Outputs &o, cudaStream_t stream);

// Haar-like window sums (k_haar.cu): the row profile's segments (warm-up)
// and the row and column taps c_a = f(a-1) - f(a), c'_B = g(B-1) - g(B).
struct HaarDev {
    int n_rs, n_rt, n_ct;
    int rs_len[4], rs_wt[4];
    int rt_a[5], rt_c[5];
    int ct_b[5], ct_c[5];
};
cudaError_t launch_haar(const Image &g, const Window &win, const HaarDev &hd, int32_t *out,
                        cudaStream_t stream);

// Window extrema (dense mn, mx planes) or, when bits != null, Bernsen's
// packed decision (k_minmax.cu).
cudaError_t launch_minmax(const Image &g, const Window &win, int32_t contrast_limit, uint8_t *mn,
                          uint8_t *mx, uint8_t *bits, int64_t out_pitch, cudaStream_t stream);

cudaError_t launch_quantile(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream);

// ---- autotuner (tune.cu) ----------------------------------------------
// A launch configuration: tile_h (0 = heuristic), edge fraction (0 =
// heuristic, 1 = uniform tiles), stripes (-1 = heuristic, 0 off, 1 on), and
// the measured microseconds per call.  The batch entry stores its window and
// quantile tile multipliers in tile_h and stripes.
struct TuneCfg {
    int32_t tile_h = 0;
    float edge = 0.0f;
    int32_t stripes = -1;
    float us = 0.0f;
};
// The configuration the launch planners of this thread use (or null): set
// for the duration of one launch by a TuneScope.
const TuneCfg *tune_override();
struct TuneScope {
    explicit TuneScope(const TuneCfg *c);
    ~TuneScope();
    TuneScope(const TuneScope &) = delete;
    TuneScope &operator=(const TuneScope &) = delete;

  private:
    const TuneCfg *prev_;
};
int tune_env();  // BZ_TUNE: -1 unset, 0 off, 1 tune on a miss
// An explicit tuning call: every tunable launch of this thread searches and
// stores its configuration while one of these lives.
struct TuneForce {
    TuneForce();
    ~TuneForce();
    TuneForce(const TuneForce &) = delete;
    TuneForce &operator=(const TuneForce &) = delete;

  private:
    bool prev_;
};
bool tune_forced();
bool tune_now(bool have);
int dim_bucket(int v);
int size_bucket(int64_t H, int64_t W);
std::string tune_key(const char *gpu, const char *kernel, int cls, int h, int w, int64_t H, int64_t W);
std::string device_tag();
bool tune_get(const std::string &key, TuneCfg &c);
void tune_put(const std::string &key, const TuneCfg &c, bool save);
std::string window_tune_key(int mode, const Window &win, int64_t rows, int64_t W);
std::string quantile_tune_key(int32_t q_num, int32_t q_den, const Window &win, int64_t H, int64_t W);
std::string batch_tune_key(int mode);
// Timed searches: `launch` runs the call once with the configuration of the
// current TuneScope; the fastest configuration goes to `best`.
bool tune_window(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1, bool pipe,
                 const std::function<cudaError_t()> &launch, cudaStream_t stream, TuneCfg &best);
bool tune_quantile(const Image &g, const Window &win, const std::function<cudaError_t()> &launch,
                   cudaStream_t stream, TuneCfg &best);

// Planner pieces the tuner reads (plan.cu, k_stripes.cu, k_quantile.cu).
int64_t one_wave_tile_rows(int64_t rows, int64_t W);
double default_edge_fraction(bool pipe);
bool stripes_allowed(int h);
int64_t quantile_band_rows(int64_t H, int64_t W, int h);
// Window-kernel plan of an H x W image on a GPU with `sms` SMs under the
// current TuneScope / environment: tile_h, edge_h, n_edge, tiles_total,
// stripes (0/1), resident warps into out[0..5].
int plan_window_launch(int64_t H, int64_t W, const Window &win, int sms, bool pipe, int64_t out[6]);

// Bounds-check status of each kernel file (bz_debug.cuh): ORs its status
// into *status, keeps the first offending address, clears it with reset;
// returns 0, 1 when the library is not a debug build, -1 on a CUDA error.
int dbg_status_window(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_small(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_stripes(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_quantile(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_minmax(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_haar(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_batch(unsigned *status, unsigned long long *addr, bool reset);
int dbg_status_table1(unsigned *status, unsigned long long *addr, bool reset);

// Stream-ordered scratch (stripe sums, global statistics, in-place bands)
// from a library-owned memory pool per device that keeps up to 256 MB
// between calls: the device's default pool returns its memory at every
// synchronisation, so a call after a synchronisation would map it again.
// Under stream capture the allocation is the graph's own (cudaMallocAsync).
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t scratch_free(void *p, cudaStream_t s);

// Library-owned per-device FP64-fallback counters: two that single-image
// calls alternate between (fallback_slot: this call's counter and the one
// its launches zero), and one for batches (fallback_counter, reset inside the
// batch graph).  bz_last_fp64_fallbacks reads the latest call's.
struct FbSlot {
    unsigned long long *use = nullptr, *clear = nullptr;
};
FbSlot fallback_slot(int device);
unsigned long long *fallback_counter(int device);
void fallback_mark_batch(int device);

// Validation helpers (return BZ_OK or an error status).
bz_status check_image(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                      int32_t w);
bz_status check_out(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                    const uint8_t *out, int64_t out_pitch);
bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb);
// Sauvola (method 0) / Niblack (1) parameters the library accepts.
bool finite_params(int method, double k, double R);

}  // namespace bz
