// Stripe pre-pass kernels: per-column window sums at the first row of every
// tile row, from which the window kernel's tiles start instead of warming up
// over the h rows above them.  The per-tile arithmetic that consumes them
// lives in bz_window.cuh (warm_from_stripes).
#include <stdlib.h>

#include "bz_internal.h"

namespace bz {

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
        return BZ_DBG_IN(rp + x, 4, g.img, dbg_image_extent(g), kDbgImage)
                   ? __ldg(reinterpret_cast<const uint32_t *>(rp + x))
                   : 0u;
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
            if (x + b < g.W && BZ_DBG_IN(out + s * g.W + x + b, 8, out, (size_t)S * g.W * 8, kDbgScratch))
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
    if (a1 - a0 <= kChunkBatch) {
        // the whole chunk in one batch of loads (one memory round trip),
        // its first rows summed apart (the branch is uniform: a warp's
        // threads share the chunk)
        uint32_t wd[kChunkBatch];
#pragma unroll
        for (int j = 0; j < kChunkBatch; j++)
            wd[j] = a0 + j < a1 ? stripe_word<VEC4>(g, a0 + j, x) : 0u;
        // four rows at a time: the bytes of each column in the four rows
        // gathered into one word (a 4 x 4 byte transpose), so that its sum
        // and its sum of squares are one DP4A each; groups before the split
        // at nm go to R, groups after it to the rest, the group across it is
        // split by a byte mask (rows past the chunk are zero words)
        const int nm = (int)(am - a0);
        uint32_t QC[4] = {0u, 0u, 0u, 0u}, QD[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int gq = 0; gq < kChunkBatch / 4; gq++) {
            const uint32_t w0 = wd[4 * gq], w1 = wd[4 * gq + 1], w2 = wd[4 * gq + 2], w3 = wd[4 * gq + 3];
            const uint32_t lo01 = __byte_perm(w0, w1, 0x5140u), hi01 = __byte_perm(w0, w1, 0x7362u);
            const uint32_t lo23 = __byte_perm(w2, w3, 0x5140u), hi23 = __byte_perm(w2, w3, 0x7362u);
            const uint32_t col[4] = {__byte_perm(lo01, lo23, 0x5410u), __byte_perm(lo01, lo23, 0x7632u),
                                     __byte_perm(hi01, hi23, 0x5410u), __byte_perm(hi01, hi23, 0x7632u)};
            const int k = nm - 4 * gq;  // rows of this group that belong to R (uniform)
            if (k >= 4) {
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    RC[b] = __dp4a(col[b], 0x01010101u, RC[b]);
                    RD[b] = __dp4a(col[b], col[b], RD[b]);
                }
            } else if (k <= 0) {
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    QC[b] = __dp4a(col[b], 0x01010101u, QC[b]);
                    QD[b] = __dp4a(col[b], col[b], QD[b]);
                }
            } else {
                const uint32_t mr = 0xFFFFFFFFu >> (8 * (4 - k));
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const uint32_t cr = col[b] & mr, cq = col[b] & ~mr;
                    RC[b] = __dp4a(cr, 0x01010101u, RC[b]);
                    RD[b] = __dp4a(cr, cr, RD[b]);
                    QC[b] = __dp4a(cq, 0x01010101u, QC[b]);
                    QD[b] = __dp4a(cq, cq, QD[b]);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 4; b++) {
            C[b] = RC[b] + QC[b];
            D[b] = RD[b] + QD[b];
        }
    } else {
        if (a0 < am)
            stripe_rows<VEC4>(g, x, a0, am, C, D);
#pragma unroll
        for (int b = 0; b < 4; b++) {
            RC[b] = C[b];
            RD[b] = D[b];
        }
        if (am < a1)
            stripe_rows<VEC4>(g, x, am, a1, C, D);
    }
#pragma unroll
    for (int b = 0; b < 4; b++)
        if (x + b < g.W && BZ_DBG_IN(QR + k * g.W + x + b, 16, QR, (size_t)K * g.W * 16, kDbgScratch))
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
            if (k + j < m && BZ_DBG_IN(QR + (s0 + k + j) * W + x, 16, QR, (size_t)(S + m + 1) * W * 16, kDbgScratch)) {
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
            const size_t qext = (size_t)(S + m + 1) * W * 16;
            rr[j] = BZ_DBG_IN(QR + (s + m) * W + x, 16, QR, qext, kDbgScratch) ? __ldg(QR + (s + m) * W + x)
                                                                              : make_uint4(0u, 0u, 0u, 0u);
            if (j > 0) {
                vin[j] = BZ_DBG_IN(QR + (s + m - 1) * W + x, 16, QR, qext, kDbgScratch)
                             ? __ldg(QR + (s + m - 1) * W + x)
                             : make_uint4(0u, 0u, 0u, 0u);
                vout[j] = BZ_DBG_IN(QR + (s - 1) * W + x, 16, QR, qext, kDbgScratch) ? __ldg(QR + (s - 1) * W + x)
                                                                                  : make_uint4(0u, 0u, 0u, 0u);
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
            if (BZ_DBG_IN(out + s * W + x, 8, out, (size_t)S * W * 8, kDbgScratch))
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

// Stripes pay off once the window spans about five tile heights: each
// tile's own warm-up reads h rows for tile_h output rows (four rows per
// step).  Measured on GB300 (4096 x 3072 page, BZ_FP64, 21-row tiles, events
// over 64 calls): 63 x 63 48.5 us without stripes, 53.1 with the chunked
// pre-pass; 255 x 255 90.5 without, 54.8 with; 31 x 127 (1.5 tile heights)
// 42.1 without.
// BZ_STRIPES=0/1 forces it (tuning), then a tuned configuration (only for
// windows of 48 rows or more, the range the pre-pass is tested on).
bool stripes_allowed(int h)
{
    return h >= 48;
}

static bool use_stripes(int h, int64_t tile_h)
{
    static const int env = [] {
        const char *e = getenv("BZ_STRIPES");
        return e ? atoi(e) : -1;
    }();
    if (env >= 0)
        return env != 0;
    const TuneCfg *t = tune_override();
    if (t && t->stripes >= 0)
        return t->stripes != 0 && stripes_allowed(h);
    return h >= 48 && h >= 5 * tile_h;
}

// Chunked form when the window spans at least two tile heights (its
// chunk sums take one round trip of loads per chunk; 63 x 63 with stripes:
// 54.7 us against 68.2 with the group form).  BZ_STRIPE_MODE=0/1 forces one
// (tuning).
static int stripe_mode(const Window &win, int64_t tile_h)
{
    static const int env_mode = [] {
        const char *e = getenv("BZ_STRIPE_MODE");
        return e ? atoi(e) : -1;
    }();
    const int m = (int)(win.h / tile_h);
    return env_mode >= 0 ? env_mode : (m >= 2 ? 1 : 0);
}

int stripe_kernel_count(const Window &win, int64_t tile_h, int64_t tiles_y)
{
    if (!use_stripes(win.h, tile_h) || tiles_y <= 1)
        return 0;
    return stripe_mode(win, tile_h) ? 2 : 1;
}

uint2 *launch_stripes(const Image &g, const Window &win, int64_t row0, int64_t tile_h,
                      int64_t tiles_y, cudaStream_t stream)
{
    if (!use_stripes(win.h, tile_h) || tiles_y <= 1)
        return nullptr;
    const int m = (int)(win.h / tile_h), hm = (int)(win.h - (int64_t)m * tile_h);
    const int mode = stripe_mode(win, tile_h);
    const bool vec4 = ((uintptr_t)g.img % 4 == 0) && (g.pitch % 4 == 0);
    const int64_t words = (g.W + 3) / 4;
    const size_t sbytes = ((size_t)tiles_y * (size_t)g.W * sizeof(uint2) + 15) & ~(size_t)15;
    const int64_t K = tiles_y + m + 1;  // chunks s .. s+m for every tile start
    const size_t qbytes = mode ? (size_t)K * (size_t)g.W * sizeof(uint4) : 0;
    uint2 *stripes = nullptr;
    if (scratch_alloc((void **)&stripes, sbytes + qbytes, stream) != cudaSuccess) {
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
            scratch_free(stripes, stream);
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
            scratch_free(stripes, stream);
            return nullptr;
        }
    }
    if (cudaGetLastError() != cudaSuccess) {
        scratch_free(stripes, stream);
        return nullptr;
    }
    return stripes;
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_stripes)

}  // namespace bz
