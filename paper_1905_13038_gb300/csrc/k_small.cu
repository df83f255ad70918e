// Small pages (a few hundred thousand pixels): the window kernel's warp tiles
// are then latency-bound (each warp walks h warm-up rows before its first
// output row), so for windows up to 63 x 63 a block computes a 32 x 64 tile
// in shared memory instead: it stages the tile plus its h-1 / w-1 halo once,
// forms the h-row column sums of every staged column (Sec. 3.1 stripe
// identity, slid down 32 rows), turns each row of column sums into running
// sums along the row, and reads every window sum as one difference of two
// running sums (the Sec. 3.1 window identity).  All sums are exact integers;
// the threshold is the certified FP32 filter with the canonical FP64 decision
// for near-ties, exactly as in the window kernel.
#include "bz_internal.h"

namespace bz {

constexpr int kSmTH = 32, kSmTW = 64, kSmThreads = 256;
constexpr int kSmMaxWin = 63;
constexpr int kSmRows = kSmTH + kSmMaxWin - 1;  // 94 staged rows at most
constexpr int kSmCols = 128;                      // >= kSmTW + kSmMaxWin - 1 = 126

template <int MODE>
__global__ void __launch_bounds__(kSmThreads)
    k_small(Image g, Window win, Thresh T, Outputs o, int64_t tiles_x, int64_t row0, int64_t row1)
{
    __shared__ uint8_t R[kSmRows][kSmCols];
    __shared__ uint32_t P1[kSmTH][kSmCols], P2[kSmTH][kSmCols];
    pdl_begin();
    fallbacks_clear(o);
    const int tid = threadIdx.x;
    const int64_t x0 = (int64_t)(blockIdx.x % tiles_x) * kSmTW;
    const int64_t y0 = row0 + (int64_t)(blockIdx.x / tiles_x) * kSmTH;
    const int h = win.h, w = win.w, l = win.l, r = win.r, oo = win.o, u = win.u;
    const int nrows = kSmTH + h - 1, ncols = kSmTW + w - 1;
    const int64_t ry0 = y0 - oo + 1, rx0 = x0 - l + 1;  // image position of R[0][0]

    // 1. stage the tile and its halo (zero outside the image)
    for (int idx = tid; idx < nrows * ncols; idx += kSmThreads) {
        const int rr = idx / ncols, cc = idx - rr * ncols;
        const int64_t gy = ry0 + rr, gx = rx0 + cc;
        R[rr][cc] = (gy >= 0 && gy < g.H && gx >= 0 && gx < g.W &&
                     BZ_DBG_IN(g.img + gy * g.pitch + gx, 1, g.img, dbg_image_extent(g), kDbgImage))
                        ? g.img[gy * g.pitch + gx]
                        : (uint8_t)0;
    }
    __syncthreads();

    // 2. column sums over h rows, slid down the 32 output rows
    for (int c = tid; c < ncols; c += kSmThreads) {
        uint32_t s1 = 0, s2 = 0;
        for (int a = 0; a < h; a++) {
            const uint32_t v = R[a][c];
            s1 += v;
            s2 += v * v;
        }
        P1[0][c] = s1;
        P2[0][c] = s2;
        for (int i = 1; i < kSmTH; i++) {
            const uint32_t vin = R[i + h - 1][c], vout = R[i - 1][c];
            s1 += vin - vout;
            s2 += vin * vin - vout * vout;
            P1[i][c] = s1;
            P2[i][c] = s2;
        }
    }
    __syncthreads();

    // 3. running sums along each row (one warp per row, 32 columns per step)
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = warp; i < kSmTH; i += kSmThreads / 32) {
        uint32_t c1 = 0, c2 = 0;
        for (int c0 = 0; c0 < ncols; c0 += 32) {
            const int c = c0 + lane;
            uint32_t v1 = c < ncols ? P1[i][c] : 0u, v2 = c < ncols ? P2[i][c] : 0u;
            v1 = warp_incl_scan<uint32_t>(v1, lane) + c1;
            v2 = warp_incl_scan<uint32_t>(v2, lane) + c2;
            if (c < ncols) {
                P1[i][c] = v1;
                P2[i][c] = v2;
            }
            c1 = __shfl_sync(0xFFFFFFFFu, v1, 31);
            c2 = __shfl_sync(0xFFFFFFFFu, v2, 31);
        }
    }
    __syncthreads();

    // 4. one output byte (8 pixels) per thread: window sums, threshold, pack
    const int i = tid >> 3, b = tid & 7;
    const int64_t gy = y0 + i, gx0 = x0 + 8 * b;
    if (gy >= row1 || gx0 >= g.W)
        return;
    const int64_t rows = (gy + u < g.H - 1 ? gy + u : g.H - 1) - (gy - oo > -1 ? gy - oo : -1);
    uint32_t byte = 0;
    unsigned long long nfb = 0;
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int jj = 8 * b + m;
        const int64_t gx = gx0 + m;
        if (gx >= g.W)
            break;
        const uint32_t S1 = P1[i][jj + w - 1] - (jj > 0 ? P1[i][jj - 1] : 0u);
        const uint32_t S2 = P2[i][jj + w - 1] - (jj > 0 ? P2[i][jj - 1] : 0u);
        const int64_t cols = (gx + r < g.W - 1 ? gx + r : g.W - 1) - (gx - l > -1 ? gx - l : -1);
        const uint32_t n = (uint32_t)(rows * cols);
        const uint32_t I = R[i + oo - 1][jj + l - 1];
        uint32_t bit;
        if (MODE == MODE_FP64_DIRECT) {
            bit = fp64_bit(T.method, I, S1, (uint64_t)S2, n, T.k, T.R);
        } else {
            const float inv_n = __frcp_rn((float)n);
            const float mu = __uint2float_rn(S1) * inv_n;
            const float var = (v_float<uint32_t>(n, (uint64_t)S2, S1) * inv_n) * inv_n;
            const float s = sqrt_approx(var);
            const float t = fmaf(fmaf(T.beta, mu, T.gamma), s, T.alpha * mu);
            const float d = t - (float)I;
            bit = __float_as_uint(d) >> 31;
            if (MODE == MODE_FP64) {
                const float mag = fmaf(fmaf(T.abeta, mu, T.agamma), s, T.aalpha * mu);
                if (fabsf(d) <= fmaf(T.eps, mag, T.delta64)) {
                    bit = fp64_bit(T.method, I, S1, (uint64_t)S2, n, T.k, T.R);
                    nfb++;
                }
            }
        }
        byte |= bit << m;
    }
    uint8_t *dst = o.bits + (gy - o.out_row0) * o.out_pitch + ((gx0 >> 3) - o.out_byte0);
    if (BZ_DBG_IN(dst, 1, o.bits, o.bits_bytes, kDbgOutput))
        *dst = (uint8_t)byte;  // padding bits stay 0
    if (MODE == MODE_FP64 && nfb && o.fallbacks)
        atomicAdd(o.fallbacks, nfb);
}

bool small_path_applies(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1)
{
    if (mode != MODE_FP64 && mode != MODE_FP32 && mode != MODE_FP64_DIRECT)
        return false;
    if (win.h > kSmMaxWin || win.w > kSmMaxWin)
        return false;
    // the window kernel's one-wave tiles would be at most 4 rows tall
    return window_tile_rows(row1 - row0, g.W, win.h, win.w) <= 4;
}

cudaError_t launch_small(int mode, const Image &g, const Window &win, const Thresh &T,
                         const Outputs &o, int64_t row0, int64_t row1, cudaStream_t stream)
{
    const int64_t tiles_x = (g.W + kSmTW - 1) / kSmTW;
    const int64_t tiles = tiles_x * ((row1 - row0 + kSmTH - 1) / kSmTH);
    if (tiles > 2147483647LL)
        return cudaErrorInvalidValue;
    switch (mode) {
    case MODE_FP64:
        return launch_pdl(k_small<MODE_FP64>, (unsigned)tiles, kSmThreads, stream, g, win, T, o, tiles_x, row0,
                          row1);
    case MODE_FP32:
        return launch_pdl(k_small<MODE_FP32>, (unsigned)tiles, kSmThreads, stream, g, win, T, o, tiles_x, row0,
                          row1);
    default:
        return launch_pdl(k_small<MODE_FP64_DIRECT>, (unsigned)tiles, kSmThreads, stream, g, win, T, o, tiles_x,
                          row0, row1);
    }
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_small)

}  // namespace bz
