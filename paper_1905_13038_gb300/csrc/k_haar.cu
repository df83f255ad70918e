// Haar-like window sums (Sec. 3.4: the recursive sums replace integral
// images for Haar-like features): for every pixel, the sum over Algorithm
// 1's h x w window of f(a) g(b) I, with f and g piecewise constant over the
// window's rows and columns (Viola and Jones's two-, three- and
// four-rectangle features are the cases with 2 or 3 segments).
//
// Recursive form.  Per column x the vertical profile sum
//   D_x(i) = sum_a f(a) I(i-o+1+a, x)
// moves down one row by D_x(i) = D_x(i-1) + sum_a c_a I(i-o+a, x), where
// c_a = f(a-1) - f(a) is non-zero only at the n_row + 1 segment boundaries
// (the Sec. 3.1 stripe identity with more than two taps).  Along the row the
// feature is sum_B c'_B P(j - l + B), P the running sum of D over the
// columns and c'_B = g(B-1) - g(B) (the window identity with more taps), so
// every pixel costs O(n_row + n_col) whatever the window size.
//
// Layout: one warp per tile of 256 output columns x 32 rows; lane k keeps D
// for the 24 consecutive columns x0 - l + 24k ... of the tile's extended
// span [x0 - l, x0 + 255 + r] (at most 767 columns) in registers; per row the
// warp turns D into P (lane prefix + warp scan) in a 3 KB shared-memory row,
// from which lane k evaluates the output columns x0 + k + 32 m.  Integer
// arithmetic is modulo 2^32; the host bounds |feature| < 2^31, so the
// result is exact.
#include "bz_internal.h"

namespace bz {

constexpr int kHaarWarps = 4;
constexpr int kHaarTileRows = 32;
constexpr int kHaarSpan = 768;  // 32 lanes x 24 columns

// 24 bytes of row `row`, columns xb .. xb+23 (zero outside [0, W)), as words.
template <bool VEC4>
__device__ __forceinline__ void haar_load24(const Image &g, int64_t row, int64_t xb, uint32_t (&v)[6])
{
    const uint8_t *rp = g.img + row * g.pitch;
    const int64_t a4 = xb >= 0 ? (xb & ~(int64_t)3) : -((-xb + 3) & ~(int64_t)3);
    if (VEC4 && a4 >= 0 && a4 + 28 <= g.W) {
        uint32_t wd[7];
        const bool ok = BZ_DBG_IN(rp + a4, 28, g.img, dbg_image_extent(g), kDbgImage);
#pragma unroll
        for (int q = 0; q < 7; q++)
            wd[q] = ok ? __ldg(reinterpret_cast<const uint32_t *>(rp + a4) + q) : 0u;
        const unsigned sh = 8u * (unsigned)(xb - a4);
#pragma unroll
        for (int q = 0; q < 6; q++)
            v[q] = __funnelshift_r(wd[q], wd[q + 1], sh);
        return;
    }
#pragma unroll
    for (int q = 0; q < 6; q++) {
        uint32_t x = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int64_t c = xb + 4 * q + b;
            if (c >= 0 && c < g.W)
                x |= (uint32_t)rp[c] << (8 * b);
        }
        v[q] = x;
    }
}

__device__ __forceinline__ void haar_acc(uint32_t (&D)[24], const uint32_t (&v)[6], int32_t c)
{
#pragma unroll
    for (int q = 0; q < 24; q++)
        D[q] += (uint32_t)c * ((v[q >> 2] >> (8 * (q & 3))) & 0xFFu);
}

template <bool VEC4>
__global__ void __launch_bounds__(32 * kHaarWarps)
    k_haar(Image g, Window win, HaarDev hd, int32_t *out, int64_t tiles_x, int64_t tiles_total)
{
    __shared__ __align__(16) uint32_t Psm[kHaarWarps][kHaarSpan];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *P = Psm[warp];
    const int64_t t = (int64_t)blockIdx.x * kHaarWarps + warp;
    if (t >= tiles_total)
        return;
    const int64_t x0 = (t % tiles_x) * 256, y0 = (t / tiles_x) * kHaarTileRows;
    const int64_t y1 = y0 + kHaarTileRows < g.H ? y0 + kHaarTileRows : g.H;
    const int64_t xb = x0 - win.l + 24 * lane;  // this lane's first span column

    // D for row y0: the whole window, segment by segment
    uint32_t D[24];
#pragma unroll
    for (int q = 0; q < 24; q++)
        D[q] = 0u;
    {
        int64_t row = y0 - win.o + 1;
#pragma unroll
        for (int s = 0; s < 4; s++) {  // constant indices: hd stays in parameter space
            const int len = s < hd.n_rs ? hd.rs_len[s] : 0;
            for (int a = 0; a < len; a++, row++) {
                if (row >= 0 && row < g.H) {
                    uint32_t v[6];
                    haar_load24<VEC4>(g, row, xb, v);
                    haar_acc(D, v, hd.rs_wt[s]);
                }
            }
        }
    }

    for (int64_t i = y0; i < y1; i++) {
        if (i > y0) {
#pragma unroll
            for (int k = 0; k < 5; k++) {
                const int64_t row = i - win.o + hd.rt_a[k];
                if (k < hd.n_rt && row >= 0 && row < g.H) {
                    uint32_t v[6];
                    haar_load24<VEC4>(g, row, xb, v);
                    haar_acc(D, v, hd.rt_c[k]);
                }
            }
        }
        // P: running sum of D over the span
        uint32_t run = 0;
        uint32_t pre[24];
#pragma unroll
        for (int q = 0; q < 24; q++) {
            run += D[q];
            pre[q] = run;
        }
        const uint32_t incl = warp_incl_scan<uint32_t>(run, lane);
        const uint32_t base = incl - run;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 24; q += 4)
            *reinterpret_cast<uint4 *>(&P[24 * lane + q]) =
                make_uint4(base + pre[q], base + pre[q + 1], base + pre[q + 2], base + pre[q + 3]);
        __syncwarp();
        // output columns x0 + lane + 32 m
#pragma unroll
        for (int m = 0; m < 8; m++) {
            const int jj = lane + 32 * m;
            if (x0 + jj < g.W) {
                uint32_t f = 0;
#pragma unroll
                for (int k = 0; k < 5; k++)
                    if (k < hd.n_ct)
                        f += (uint32_t)hd.ct_c[k] * P[jj + hd.ct_b[k]];
                if (BZ_DBG_IN(out + i * g.W + x0 + jj, 4, out, (size_t)(g.H * g.W) * 4, kDbgOutput))
                    out[i * g.W + x0 + jj] = (int32_t)f;
            }
        }
    }
}

cudaError_t launch_haar(const Image &g, const Window &win, const HaarDev &hd, int32_t *out,
                        cudaStream_t stream)
{
    const int64_t tiles_x = (g.W + 255) / 256;
    const int64_t tiles = tiles_x * ((g.H + kHaarTileRows - 1) / kHaarTileRows);
    const int64_t blocks = (tiles + kHaarWarps - 1) / kHaarWarps;
    if (blocks > 2147483647LL)
        return cudaErrorInvalidValue;
    const bool vec4 = ((uintptr_t)g.img % 4 == 0) && (g.pitch % 4 == 0);
    if (vec4)
        k_haar<true><<<(unsigned)blocks, 32 * kHaarWarps, 0, stream>>>(g, win, hd, out, tiles_x, tiles);
    else
        k_haar<false><<<(unsigned)blocks, 32 * kHaarWarps, 0, stream>>>(g, win, hd, out, tiles_x, tiles);
    return cudaGetLastError();
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_haar)

}  // namespace bz
