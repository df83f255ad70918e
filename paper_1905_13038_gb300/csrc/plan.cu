// Host-side planning of the window kernel's launches: the one-wave tile
// height, the balanced tile schedule (shorter edge tiles), the tuning
// switches read from the environment, and the library's stream-ordered
// scratch pool.  Pure host code; the kernels that consume the schedule live
// in k_window.cu and k_table1.cu.
#include <stdlib.h>

#include <mutex>

#include "bz_internal.h"

namespace bz {

bool pdl_enabled()
{
    static const bool on = [] {
        const char *e = getenv("BZ_PDL");
        return !(e && atoi(e) == 0);
    }();
    return on;
}

// Warps resident at once on this device (one wave of k_window).
static int64_t resident_warps()
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int64_t)sms * kBlocksPerSM * kWarpsPerBlock;
}

// The shortest tile height for which every 256-column warp tile of an
// H x W image is resident at once with `resident` warps.
static int64_t one_wave_rows(int64_t H, int64_t W, int64_t resident)
{
    const int64_t tiles_x = (W + kTileCols - 1) / kTileCols;
    int64_t bands = resident / tiles_x;
    if (bands < 1)
        bands = 1;
    int64_t th = (H + bands - 1) / bands;
    if (th < 1)
        th = 1;
    return th;
}

int64_t one_wave_tile_rows(int64_t rows, int64_t W)
{
    return one_wave_rows(rows, W, resident_warps());
}

// One wave of warp tiles: the shortest tiles for which every tile of the
// image is resident at once (SMs x 4 blocks x 4 warps).  Measured on GB300:
// on the 4096 x 3072 page this gives 21 rows (8 % faster than 24, while 20
// rows spills into a second wave); on small pages it gives 1-4 rows, which
// halves the latency (the launch is latency-bound and every warp's work
// shrinks).  BZ_TILE_ROWS overrides it, then a tuned configuration.
static int64_t tile_rows_for(int64_t H, int64_t W, int64_t resident)
{
    static const int64_t env = [] {
        const char *e = getenv("BZ_TILE_ROWS");
        return e ? (int64_t)atoll(e) : (int64_t)0;
    }();
    if (env > 0)
        return env < H ? env : H;
    const TuneCfg *t = tune_override();
    if (t && t->tile_h > 0)
        return t->tile_h < H ? t->tile_h : H;
    return one_wave_rows(H, W, resident);
}

int64_t window_tile_rows(int64_t H, int64_t W, int h, int w)
{
    (void)h;
    (void)w;
    return tile_rows_for(H, W, resident_warps());
}

// Edge-tile height as a fraction of the interior height: the measured time
// per row of an edge tile is above an interior row's on the pipelined path
// (clamped streams, per-column counts) and 1.3-2x on the generic path
// (GB300, 4096 x 3072 page).  Pipelined path, Sauvola BZ_FP64 at 15², 63²,
// 31 x 127 (events over 64 calls each, with the column-sum warm-up): 0.6 gave
// 32.5 / 43.1 / 39.7 us, 0.7 33.3 / 42.6 / 38.4, 0.82 36.9 / 42.7 / 39.5,
// uniform tiles 39.5 / 45.9 / 42.5.  Table 1 methods (generic path), Wolf /
// Rais / Phansalkar at 15², 31², 63²: 0.5 gave 778 us summed over the nine
// calls, 0.6 788, 0.7 795, uniform tiles 940.  BZ_EDGE_FRAC overrides it
// (tuning; >= 1 disables the balanced schedule).
double default_edge_fraction(bool pipe)
{
    return pipe ? 0.7 : 0.5;
}

static double edge_fraction(bool pipe)
{
    static const double env = [] {
        const char *e = getenv("BZ_EDGE_FRAC");
        return e ? atof(e) : 0.0;
    }();
    if (env > 0.0)
        return env;
    const TuneCfg *t = tune_override();
    if (t && t->edge > 0.0f)
        return t->edge;
    return default_edge_fraction(pipe);
}

// The schedule of rows [row0, row1) of a W-column image from its one-wave
// tile height: uniform, or, without stripe warm-up and with at least three
// tile columns, the shortest interior tiles (at most two rows taller than
// the uniform ones) whose grid, with edge tiles of f times their height,
// still fits in `resident` warps (pure host arithmetic).
static TileSched plan_sched(int64_t row0, int64_t row1, int64_t W, int64_t tile_h, int64_t resident, double f,
                            bool stripes)
{
    TileSched S;
    const int64_t rows = row1 - row0;
    S.tiles_x = (W + kTileCols - 1) / kTileCols;
    S.tile_h = tile_h;
    S.edge_h = tile_h;
    S.n_edge = 0;
    S.row0 = row0;
    S.row1 = row1;
    S.tx0 = 0;
    S.prefetch = 0;
    const int64_t uniform = S.tiles_x * ((rows + tile_h - 1) / tile_h);
    S.tiles_total = uniform;
    if (!stripes && S.tiles_x >= 3 && f < 1.0 && tile_h > 4) {
        const int64_t cap = uniform > resident ? uniform : resident;
        for (int64_t th = tile_h; th <= tile_h + 2; th++) {
            int64_t eh = (int64_t)((double)th * f + 0.5);
            eh = eh < 1 ? 1 : eh;
            const int64_t ne = 2 * ((rows + eh - 1) / eh);
            const int64_t total = ne + (S.tiles_x - 2) * ((rows + th - 1) / th);
            if (eh < th && total <= cap) {
                S.tile_h = th;
                S.edge_h = eh;
                S.n_edge = ne;
                S.tiles_total = total;
                break;
            }
        }
    }
    return S;
}

// The tile schedule of a launch over rows [row0, row1) (plan_sched with this
// device's resident warps and the tuning overrides).
TileSched make_sched(const Image &g, const Window &win, int64_t row0, int64_t row1, bool pipe,
                     bool stripes)
{
    TileSched S = plan_sched(row0, row1, g.W, window_tile_rows(row1 - row0, g.W, win.h, win.w),
                             resident_warps(), edge_fraction(pipe), stripes);
    // without stripes the image is usually not in L2 yet (the stripe
    // pre-pass has just read it otherwise).  BZ_PREFETCH=0 turns it off.
    static const bool pf = [] {
        const char *e = getenv("BZ_PREFETCH");
        return !(e && atoi(e) == 0);
    }();
    S.prefetch = (pf && !stripes) ? 1 : 0;
    return S;
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {nullptr};
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess)
        return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (cap != cudaStreamCaptureStatusNone || dev < 0 || dev >= 64)
        return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            if (cudaMemPoolCreate(&np, &props) == cudaSuccess) {
                uint64_t keep = 256ull << 20;
                cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
                pools[dev] = np;
            } else {
                cudaGetLastError();
            }
        }
        pool = pools[dev];
    }
    if (!pool)
        return cudaMallocAsync(p, bytes, s);
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t scratch_free(void *p, cudaStream_t s)
{
    return cudaFreeAsync(p, s);
}

int plan_window_launch(int64_t H, int64_t W, const Window &win, int sms, bool pipe, int64_t out[6])
{
    if (H < 1 || W < 1 || sms < 1)
        return -1;
    const int64_t resident = (int64_t)sms * kBlocksPerSM * kWarpsPerBlock;
    const int64_t th = tile_rows_for(H, W, resident);
    const int64_t tiles_y = (H + th - 1) / th;
    const bool st = stripe_kernel_count(win, th, tiles_y) > 0;
    const TileSched S = plan_sched(0, H, W, th, resident, edge_fraction(pipe), st);
    out[0] = S.tile_h;
    out[1] = S.edge_h;
    out[2] = S.n_edge;
    out[3] = S.tiles_total;
    out[4] = st ? 1 : 0;
    out[5] = resident;
    return 0;
}

// Pure form for planning and tests: the schedule on a GPU with `sms` SMs.
int plan_tile_schedule(int64_t H, int64_t W, int sms, bool pipe, bool stripes, int64_t out[6])
{
    if (H < 1 || W < 1 || sms < 1)
        return -1;
    const int64_t resident = (int64_t)sms * kBlocksPerSM * kWarpsPerBlock;
    const TileSched S =
        plan_sched(0, H, W, one_wave_rows(H, W, resident), resident, default_edge_fraction(pipe), stripes);
    out[0] = S.tiles_x;
    out[1] = S.tile_h;
    out[2] = S.edge_h;
    out[3] = S.n_edge;
    out[4] = S.tiles_total;
    out[5] = resident;
    return 0;
}

}  // namespace bz
