// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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
// The same over the output rows [row0, row1) only (windows still see the
// whole image).
// Kernels one launch_window_rows call enqueues (stripe pre-pass included).
int window_kernel_count(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1);
cudaError_t launch_window_rows(int mode, const Image &g, const Window &win, const Thresh &T,
                               const Outputs &o, int64_t row0, int64_t row1, cudaStream_t stream);

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

// Library-owned per-device scratch: FP64-fallback counter.
unsigned long long *fallback_counter(int device);

// Validation helpers (return BZ_OK or an error status).
bz_status check_image(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch, int32_t h,
                      int32_t w);
bz_status check_out(const uint8_t *image, int64_t H, int64_t W, int64_t in_pitch,
                    const uint8_t *out, int64_t out_pitch);
bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb);

}  // namespace bz
