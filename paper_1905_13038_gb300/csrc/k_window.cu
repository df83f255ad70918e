// Window-statistics kernels: Sauvola / Niblack binarization (FP64-exact,
// FP32, FP64-direct), the exact window-sum export and the FP32-vs-FP64
// report.  The per-tile arithmetic lives in bz_window.cuh.
#include <math.h>
#include <stdlib.h>

#include "bz_internal.h"

namespace bz {

constexpr int kWarpsPerBlock = 4;
constexpr int kBlocksPerSM = 4;  // 128 registers per thread

// The tiles of one launch.  Edge tiles (the first and last tile columns)
// clamp their byte streams and look up per-column counts, so they take
// longer per row; with a one-wave grid the slowest warps set the launch's
// duration.  A balanced schedule therefore gives the two edge columns
// shorter tiles (edge_h < tile_h rows) and lists them first (n_edge tiles,
// alternating left and right column); the uniform schedule has n_edge = 0
// and every column in the tile_h grid.
struct TileSched {
    int64_t tiles_x, tile_h, edge_h, n_edge, tiles_total, row0, row1;
    int prefetch;  // tiles start with an L2 prefetch of their input
};

// AW > 0: every tile takes the pipelined path with AW anchor words per lane
// (the host checked pipe_words); the variants are separate kernels so that
// each gets its own register allocation.  `stripes` (uniform schedules only):
// column sums at the first row of every tile row.
template <int MODE, bool VEC, typename S2T, bool WARMB, int AW>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kBlocksPerSM)
    k_window(Image g, Window win, Thresh T, Outputs o, TileSched S, const uint2 *stripes)
{
    __shared__ uint4 slots[kWarpsPerBlock][AW ? 384 : 1];  // 6 KB per warp (pipelined path)
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock;
    // tile t: column tx, rows [y0, y1), stripe sums st
    auto tile_of = [&](int64_t t, int64_t &tx, int64_t &y0, int64_t &y1, const uint2 *&st) {
        st = nullptr;
        if (t < S.n_edge) {
            tx = (t & 1) ? S.tiles_x - 1 : 0;
            y0 = S.row0 + (t >> 1) * S.edge_h;
            y1 = y0 + S.edge_h;
        } else {
            const int64_t t2 = t - S.n_edge;
            const int64_t ncol = S.n_edge ? S.tiles_x - 2 : S.tiles_x;
            const int64_t ty = t2 / ncol;
            tx = (S.n_edge ? 1 : 0) + (t2 - ty * ncol);
            y0 = S.row0 + ty * S.tile_h;
            y1 = y0 + S.tile_h;
            if (stripes)
                st = stripes + ty * g.W;
        }
        if (y1 > S.row1)
            y1 = S.row1;
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
    return T;
}

// Stripe pre-pass.  A tile's warm-up re-reads the h window rows above its
// first output row, so each image row is warmed ~h / tile_h times; for tall
// windows that dominates.  This kernel computes, once per column, the column
// sums C = sum I and D = sum I^2 over the window rows of every tile's first
// row (the Sec. 3.1 stripe identity, slid down the column), so that a tile
// starts from them (warm_from_stripes).  One thread owns 4 columns and
// `group` consecutive tile starts: it sums the h rows of the first,
// then slides tile_h rows at a time (one row in, one row out) to the next.
constexpr int kStripeThreads = 128;
constexpr int kStripeBatch = 16;  // rows whose loads are issued together

template <bool VEC4>
__device__ __forceinline__ uint32_t stripe_word(const Image &g, int64_t row, int64_t x)
{
    const uint8_t *rp = g.img + row * g.pitch;
    if (VEC4 && x + 4 <= g.W)
        return __ldg(reinterpret_cast<const uint32_t *>(rp + x));
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; b++)
        if (x + b < g.W)
            v |= (uint32_t)rp[x + b] << (8 * b);
    return v;
}

__device__ __forceinline__ void stripe_acc(uint32_t (&C)[4], uint32_t (&D)[4], uint32_t wd, int sign)
{
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const uint32_t v = (wd >> (8 * b)) & 0xFFu;
        C[b] += (uint32_t)sign * v;
        D[b] += (uint32_t)sign * v * v;
    }
}

template <bool VEC4>
__global__ void __launch_bounds__(kStripeThreads)
    k_stripes(Image g, int o, int u, int64_t row0, int64_t tile_h, int64_t S, int64_t words,
              int group, uint2 *out)
{
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * kStripeThreads + threadIdx.x;
    const int64_t q = t % words, s0 = (t / words) * group;
    if (s0 >= S)
        return;
    const int64_t s1 = s0 + group < S ? s0 + group : S;
    const int64_t x = 4 * q;
    uint32_t C[4] = {0u, 0u, 0u, 0u}, D[4] = {0u, 0u, 0u, 0u};
    auto store = [&](int64_t s) {
#pragma unroll
        for (int b = 0; b < 4; b++)
            if (x + b < g.W)
                out[s * g.W + x + b] = make_uint2(C[b], D[b]);
    };
    // window rows (y - o, y + u] of the first tile start y, eight loads at a time
    const int64_t y = row0 + s0 * tile_h;
    int64_t a_lo = y - o + 1, a_hi = y + u;
    if (a_lo < 0)
        a_lo = 0;
    if (a_hi > g.H - 1)
        a_hi = g.H - 1;
    for (int64_t a = a_lo; a <= a_hi; a += kStripeBatch) {
        uint32_t wd[kStripeBatch];
#pragma unroll
        for (int k = 0; k < kStripeBatch; k++)
            wd[k] = a + k <= a_hi ? stripe_word<VEC4>(g, a + k, x) : 0u;
#pragma unroll
        for (int k = 0; k < kStripeBatch; k++)
            stripe_acc(C, D, wd[k], 1);
    }
    store(s0);
    // slide to the next tile starts: rows y' + u enter, rows y' - o leave
    for (int64_t s = s0 + 1; s < s1; s++) {
        const int64_t ys = row0 + s * tile_h;
        for (int64_t yy = ys - tile_h + 1; yy <= ys; yy += kStripeBatch / 2) {
            uint32_t win_[kStripeBatch / 2], wout[kStripeBatch / 2];
#pragma unroll
            for (int k = 0; k < kStripeBatch / 2; k++) {
                const int64_t r = yy + k;
                win_[k] = (r <= ys && r + u < g.H) ? stripe_word<VEC4>(g, r + u, x) : 0u;
                wout[k] = (r <= ys && r - o >= 0) ? stripe_word<VEC4>(g, r - o, x) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kStripeBatch / 2; k++) {
                stripe_acc(C, D, win_[k], 1);
                stripe_acc(C, D, wout[k], -1);
            }
        }
        store(s);
    }
}

// Chunked form of the same pre-pass.  With p_k = row0 - o + 1 + k tile_h, the
// window rows of tile start s are [p_s, p_s + h) = chunks s .. s+m-1 plus the
// first h - m tile_h rows of chunk s+m (m = floor(h / tile_h)).  Phase 1 sums
// every chunk (Q_k) and its first h - m tile_h rows (R_k) in parallel, each
// image row read once per column; phase 2 slides a window of m chunk sums down
// each column: C(s) = sum_{k=s}^{s+m-1} Q_k + R_{s+m}.
// Column sums of 4 columns over a run of rows, packed: the sums of columns
// 0 and 2 (lo) and 1 and 3 (hi) in 16-bit halves, valid for up to 257 rows;
// the sums of squares per column (one dp4a each, the word times the word
// with one byte kept).
struct PackedSums {
    uint32_t lo = 0u, hi = 0u, d[4] = {0u, 0u, 0u, 0u};
    __device__ __forceinline__ void add(uint32_t wd)
    {
        lo += wd & 0x00FF00FFu;
        hi += (wd >> 8) & 0x00FF00FFu;
#pragma unroll
        for (int b = 0; b < 4; b++)
            d[b] = __dp4a(wd, wd & (0xFFu << (8 * b)), d[b]);
    }
    // move the packed column sums into 32-bit C and reset them
    __device__ __forceinline__ void flush(uint32_t (&C)[4])
    {
        C[0] += lo & 0xFFFFu;
        C[2] += lo >> 16;
        C[1] += hi & 0xFFFFu;
        C[3] += hi >> 16;
        lo = hi = 0u;
    }
};

// Sums of the rows [r0, r1) (inside the image) of the 4 columns at x into
// C (flushed) and D.  The loads of up to kChunkBatch rows are issued
// together (the pre-pass is bound by memory latency: one round trip per
// batch), the rows past r1 predicated off.
constexpr int kChunkBatch = 24;

template <bool VEC4>
__device__ __forceinline__ void stripe_rows(const Image &g, int64_t x, int64_t r0, int64_t r1, uint32_t (&C)[4],
                                            uint32_t (&D)[4])
{
    PackedSums P;
    int run = 0;  // rows in the packed sums (flushed at 240 < 257)
    for (int64_t r = r0; r < r1; r += kChunkBatch) {
        uint32_t wd[kChunkBatch];
#pragma unroll
        for (int j = 0; j < kChunkBatch; j++)
            wd[j] = r + j < r1 ? stripe_word<VEC4>(g, r + j, x) : 0u;
#pragma unroll
        for (int j = 0; j < kChunkBatch; j++)
            P.add(wd[j]);
        run += kChunkBatch;
        if (run >= 240) {
            P.flush(C);
            run = 0;
        }
    }
    P.flush(C);
#pragma unroll
    for (int b = 0; b < 4; b++)
        D[b] += P.d[b];
}

template <bool VEC4>
__global__ void __launch_bounds__(kStripeThreads)
    k_stripe_chunks(Image g, int64_t p0, int64_t tile_h, int hm, int64_t K, int64_t words,
                    uint4 *QR)
{
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * kStripeThreads + threadIdx.x;
    const int64_t q = t % words, k = t / words;
    if (k >= K)
        return;
    const int64_t x = 4 * q;
    // chunk rows [pk, pk + tile_h) and its first hm rows, clipped to the
    // image (rows outside it are zero)
    const int64_t pk = p0 + k * tile_h;
    const int64_t a0 = pk > 0 ? pk : 0;
    const int64_t a1 = pk + tile_h < g.H ? pk + tile_h : g.H;
    int64_t am = pk + hm;
    am = am < a0 ? a0 : (am > a1 ? a1 : am);
    uint32_t C[4] = {0u, 0u, 0u, 0u}, D[4] = {0u, 0u, 0u, 0u};
    uint32_t RC[4] = {0u, 0u, 0u, 0u}, RD[4] = {0u, 0u, 0u, 0u};
    if (a0 < am)
        stripe_rows<VEC4>(g, x, a0, am, C, D);
#pragma unroll
    for (int b = 0; b < 4; b++) {
        RC[b] = C[b];
        RD[b] = D[b];
    }
    if (am < a1)
        stripe_rows<VEC4>(g, x, am, a1, C, D);
#pragma unroll
    for (int b = 0; b < 4; b++)
        if (x + b < g.W)
            QR[k * g.W + x + b] = make_uint4(C[b], D[b], RC[b], RD[b]);
}

// Phase 2: one thread per column and G consecutive tile starts; the loads of
// its G starts are independent of the running sums, so they are issued
// together.
template <int G>
__global__ void __launch_bounds__(kStripeThreads)
    k_stripe_slide(int64_t W, int64_t S, int m, const uint4 *QR, uint2 *out)
{
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * kStripeThreads + threadIdx.x;
    const int64_t x = t % W, s0 = (t / W) * G;
    if (s0 >= S)
        return;
    uint32_t c = 0, d = 0;
    for (int k = 0; k < m; k += 16) {  // 16 chunk sums per round trip
        uint2 v[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            v[j] = make_uint2(0u, 0u);
            if (k + j < m) {
                const uint4 q = __ldg(QR + (s0 + k + j) * W + x);
                v[j] = make_uint2(q.x, q.y);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; j++) {
            c += v[j].x;
            d += v[j].y;
        }
    }
    uint4 vin[G], vout[G], rr[G];
#pragma unroll
    for (int j = 0; j < G; j++) {
        const int64_t s = s0 + j;
        if (s < S) {
            rr[j] = __ldg(QR + (s + m) * W + x);
            if (j > 0) {
                vin[j] = __ldg(QR + (s + m - 1) * W + x);
                vout[j] = __ldg(QR + (s - 1) * W + x);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < G; j++) {
        const int64_t s = s0 + j;
        if (s < S) {
            if (j > 0) {
                c += vin[j].x - vout[j].x;
                d += vin[j].y - vout[j].y;
            }
            out[s * W + x] = make_uint2(c + rr[j].z, d + rr[j].w);
        }
    }
}

// Tile starts per pre-pass thread: fewer means more threads (latency
// hiding) but more repeated h-row sums (BZ_STRIPE_GROUP overrides: tuning).
static int stripe_group()
{
    static const int env = [] {
        const char *e = getenv("BZ_STRIPE_GROUP");
        return e ? atoi(e) : 0;
    }();
    return env > 0 ? env : 2;
}

// Windows at least this tall start their tiles from the stripe pre-pass
// (measured on GB300; BZ_STRIPES=0/1 forces it off/on).
// Stripes pay off once the window spans about five tile heights: each tile's
// own warm-up reads h rows for tile_h output rows.  Measured on GB300 (4096 x
// 3072 page, 21-row tiles): 63 x 63 64 us per call without stripes (the edge
// columns then also get the balanced schedule) against 88 us with them;
// 255 x 255 143 us without against 78 us with.  BZ_STRIPES=0/1 forces it
// (tuning).
static bool use_stripes(int h, int64_t tile_h)
{
    static const int env = [] {
        const char *e = getenv("BZ_STRIPES");
        return e ? atoi(e) : -1;
    }();
    if (env >= 0)
        return env != 0;
    return h >= 48 && h >= 5 * tile_h;
}

uint2 *launch_stripes(const Image &g, const Window &win, int64_t row0, int64_t tile_h,
                      int64_t tiles_y, cudaStream_t stream)
{
    if (!use_stripes(win.h, tile_h) || tiles_y <= 1)
        return nullptr;
    // chunked form when the window spans at least four tile heights (measured
    // on GB300: 255 x 255 86 vs 105 us; at 63 x 63, three tile heights, the
    // per-group slide is 2 us faster).  BZ_STRIPE_MODE=0/1 forces one (tuning).
    static const int env_mode = [] {
        const char *e = getenv("BZ_STRIPE_MODE");
        return e ? atoi(e) : -1;
    }();
    const int m = (int)(win.h / tile_h), hm = (int)(win.h - (int64_t)m * tile_h);
    const int mode = env_mode >= 0 ? env_mode : (m >= 4 ? 1 : 0);
    const bool vec4 = ((uintptr_t)g.img % 4 == 0) && (g.pitch % 4 == 0);
    const int64_t words = (g.W + 3) / 4;
    const size_t sbytes = ((size_t)tiles_y * (size_t)g.W * sizeof(uint2) + 15) & ~(size_t)15;
    const int64_t K = tiles_y + m + 1;  // chunks s .. s+m for every tile start
    const size_t qbytes = mode ? (size_t)K * (size_t)g.W * sizeof(uint4) : 0;
    uint2 *stripes = nullptr;
    if (cudaMallocAsync((void **)&stripes, sbytes + qbytes, stream) != cudaSuccess) {
        cudaGetLastError();  // no scratch: the tiles warm up themselves
        return nullptr;
    }
    const int group = stripe_group();
    if (mode) {
        uint4 *QR = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(stripes) + sbytes);
        const int64_t p0 = row0 - win.o + 1;
        const int64_t b1 = (words * K + kStripeThreads - 1) / kStripeThreads;
        cudaError_t e = vec4 ? launch_pdl(k_stripe_chunks<true>, (unsigned)b1, kStripeThreads, stream, g, p0,
                                          tile_h, hm, K, words, QR)
                             : launch_pdl(k_stripe_chunks<false>, (unsigned)b1, kStripeThreads, stream, g, p0,
                                          tile_h, hm, K, words, QR);
        constexpr int sg = 8;  // tile starts per sliding thread
        const int64_t b2 = (g.W * ((tiles_y + sg - 1) / sg) + kStripeThreads - 1) / kStripeThreads;
        if (e == cudaSuccess)
            e = launch_pdl(k_stripe_slide<sg>, (unsigned)b2, kStripeThreads, stream, g.W, tiles_y, m,
                           (const uint4 *)QR, stripes);
        if (e != cudaSuccess) {
            cudaFreeAsync(stripes, stream);
            return nullptr;
        }
    } else {
        const int64_t threads = words * ((tiles_y + group - 1) / group);
        const int64_t sblocks = (threads + kStripeThreads - 1) / kStripeThreads;
        const cudaError_t e =
            vec4 ? launch_pdl(k_stripes<true>, (unsigned)sblocks, kStripeThreads, stream, g, win.o, win.u, row0,
                              tile_h, tiles_y, words, group, stripes)
                 : launch_pdl(k_stripes<false>, (unsigned)sblocks, kStripeThreads, stream, g, win.o, win.u,
                              row0, tile_h, tiles_y, words, group, stripes);
        if (e != cudaSuccess) {
            cudaFreeAsync(stripes, stream);
            return nullptr;
        }
    }
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(stripes, stream);
        return nullptr;
    }
    return stripes;
}

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

int64_t window_tile_rows(int64_t H, int64_t W, int h, int w)
{
    (void)h;
    (void)w;
    // One wave of warp tiles: the shortest tiles for which every tile of the
    // image is resident at once (SMs x 4 blocks x 4 warps).  Measured on
    // GB300: on the 4096 x 3072 page this gives 21 rows (8 % faster than 24,
    // while 20 rows spills into a second wave); on small pages it gives
    // 1-4 rows, which halves the latency (the launch is latency-bound and
    // every warp's work shrinks).  BZ_TILE_ROWS overrides it (tuning).
    static const int64_t env = [] {
        const char *e = getenv("BZ_TILE_ROWS");
        return e ? (int64_t)atoll(e) : (int64_t)0;
    }();
    if (env > 0)
        return env < H ? env : H;
    const int64_t tiles_x = (W + kTileCols - 1) / kTileCols;
    int64_t bands = resident_warps() / tiles_x;
    if (bands < 1)
        bands = 1;
    int64_t th = (H + bands - 1) / bands;
    if (th < 1)
        th = 1;
    return th;
}

// Edge-tile height as a fraction of the interior height: the measured time
// per row of an edge tile is about 1.2x an interior row's on the pipelined
// path and 1.3-2x on the generic path (GB300, 4096 x 3072 page).
// BZ_EDGE_FRAC overrides it (tuning; >= 1 disables the balanced schedule).
static double edge_fraction(bool pipe)
{
    static const double env = [] {
        const char *e = getenv("BZ_EDGE_FRAC");
        return e ? atof(e) : 0.0;
    }();
    if (env > 0.0)
        return env;
    return pipe ? 0.82 : 0.7;
}

// The tile schedule of a launch over rows [row0, row1): one-wave interior
// tiles, and for launches without stripe warm-up and with at least three
// tile columns, shorter edge tiles as long as the whole grid stays one wave.
static TileSched make_sched(const Image &g, const Window &win, int64_t row0, int64_t row1, bool pipe,
                            bool stripes)
{
    TileSched S;
    const int64_t rows = row1 - row0;
    S.tiles_x = (g.W + kTileCols - 1) / kTileCols;
    S.tile_h = window_tile_rows(rows, g.W, win.h, win.w);
    S.edge_h = S.tile_h;
    S.n_edge = 0;
    S.row0 = row0;
    S.row1 = row1;
    // without stripes the image is usually not in L2 yet (the stripe
    // pre-pass has just read it otherwise).  BZ_PREFETCH=0 turns it off.
    static const bool pf = [] {
        const char *e = getenv("BZ_PREFETCH");
        return !(e && atoi(e) == 0);
    }();
    S.prefetch = (pf && !stripes) ? 1 : 0;
    const int64_t uniform = S.tiles_x * ((rows + S.tile_h - 1) / S.tile_h);
    S.tiles_total = uniform;
    const double f = edge_fraction(pipe);
    if (!stripes && S.tiles_x >= 3 && f < 1.0 && S.tile_h > 4) {
        // the shortest interior tiles (at most two rows taller than the
        // uniform ones) whose grid, with edge tiles of f times their height,
        // still fits in one wave
        const int64_t cap = uniform > resident_warps() ? uniform : resident_warps();
        for (int64_t th = S.tile_h; th <= S.tile_h + 2; th++) {
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

template <int MODE, bool VEC, typename S2T, bool WARMB>
static cudaError_t launch_t(const Image &g, const Window &win, const Thresh &T, const Outputs &o,
                            int64_t row0, int64_t row1, cudaStream_t stream)
{
    constexpr bool kCanPipe = VEC && (MODE == MODE_FP64 || MODE == MODE_FP32) && sizeof(S2T) == 4;
    const int aw = kCanPipe ? pipe_words(MODE, VEC, sizeof(S2T) == 4, g, win) : 0;
    const bool pipe = aw > 0;
    const int64_t tile_h0 = window_tile_rows(row1 - row0, g.W, win.h, win.w);
    const int64_t tiles_y0 = (row1 - row0 + tile_h0 - 1) / tile_h0;
    uint2 *stripes = launch_stripes(g, win, row0, tile_h0, tiles_y0, stream);
    const TileSched S = make_sched(g, win, row0, row1, pipe, stripes != nullptr);
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
    if (stripes && cudaFreeAsync(stripes, stream) != cudaSuccess && e == cudaSuccess)
        e = cudaGetLastError();
    return e;
}

template <int MODE>
static cudaError_t launch_m(const Image &g, const Window &win, const Thresh &T, const Outputs &o,
                            int64_t row0, int64_t row1, cudaStream_t stream)
{
    if (small_path_applies(MODE, g, win, row0, row1))
        return launch_small(MODE, g, win, T, o, row0, row1, stream);
    const bool vec = ((uintptr_t)g.img % 8 == 0) && (g.pitch % 8 == 0);
    const bool wide = (int64_t)win.h * win.w > 66051;  // S2 may reach 2^32
    // short tiles (a small image): the launch is latency-bound, so the
    // warm-up issues its loads in batches (binarize modes only)
    static const int env_warmb = [] {  // BZ_WARMB=0/1 forces it (tuning)
        const char *e = getenv("BZ_WARMB");
        return e ? atoi(e) : -1;
    }();
    const bool warmb = (MODE == MODE_FP64 || MODE == MODE_FP32) &&
                       (env_warmb >= 0 ? env_warmb != 0
                                       : window_tile_rows(row1 - row0, g.W, win.h, win.w) <= 4);
    constexpr bool kB = (MODE == MODE_FP64 || MODE == MODE_FP32);
    if (warmb) {
        if (vec)
            return wide ? launch_t<MODE, true, unsigned long long, kB>(g, win, T, o, row0, row1, stream)
                        : launch_t<MODE, true, uint32_t, kB>(g, win, T, o, row0, row1, stream);
        return wide ? launch_t<MODE, false, unsigned long long, kB>(g, win, T, o, row0, row1, stream)
                    : launch_t<MODE, false, uint32_t, kB>(g, win, T, o, row0, row1, stream);
    }
    if (vec)
        return wide ? launch_t<MODE, true, unsigned long long, false>(g, win, T, o, row0, row1, stream)
                    : launch_t<MODE, true, uint32_t, false>(g, win, T, o, row0, row1, stream);
    return wide ? launch_t<MODE, false, unsigned long long, false>(g, win, T, o, row0, row1, stream)
                : launch_t<MODE, false, uint32_t, false>(g, win, T, o, row0, row1, stream);
}

cudaError_t launch_window_rows(int mode, const Image &g, const Window &win, const Thresh &T,
                               const Outputs &o, int64_t row0, int64_t row1, cudaStream_t stream)
{
    if (row0 < 0 || row1 > g.H || row0 >= row1)
        return cudaErrorInvalidValue;
    switch (mode) {
    case MODE_FP64: return launch_m<MODE_FP64>(g, win, T, o, row0, row1, stream);
    case MODE_FP32: return launch_m<MODE_FP32>(g, win, T, o, row0, row1, stream);
    case MODE_FP64_DIRECT: return launch_m<MODE_FP64_DIRECT>(g, win, T, o, row0, row1, stream);
    case MODE_SUMS: return launch_m<MODE_SUMS>(g, win, T, o, row0, row1, stream);
    case MODE_REPORT: return launch_m<MODE_REPORT>(g, win, T, o, row0, row1, stream);
    default: return cudaErrorInvalidValue;
    }
}

int window_kernel_count(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1)
{
    if (small_path_applies(mode, g, win, row0, row1))
        return 1;
    const int64_t tile_h = window_tile_rows(row1 - row0, g.W, win.h, win.w);
    const int64_t tiles_y = (row1 - row0 + tile_h - 1) / tile_h;
    if (!use_stripes(win.h, tile_h) || tiles_y <= 1)
        return 1;
    static const int env_mode = [] {
        const char *e = getenv("BZ_STRIPE_MODE");
        return e ? atoi(e) : -1;
    }();
    const int m = (int)(win.h / tile_h);
    return (env_mode >= 0 ? env_mode : (m >= 4 ? 1 : 0)) ? 3 : 2;
}

cudaError_t launch_window(int mode, const Image &g, const Window &win, const Thresh &T,
                          const Outputs &o, cudaStream_t stream)
{
    return launch_window_rows(mode, g, win, T, o, 0, g.H, stream);
}

}  // namespace bz
