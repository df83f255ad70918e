// Local minimum and maximum of the clipped window (Sec. 3.4: Bernsen's
// midrange and the local contrast), and Bernsen binarization.
//
// The paper keeps the extrema recursively with deques.  A deque is a
// sequential, data-dependent structure; on the GPU the same Theta(1)-per-
// pixel bound comes from splitting every window at a fixed row (van Herk /
// Gil-Werman): a CTA owns a tile of TW output columns x TR output rows and
//  1. vertical: for a segment of rows [a, b) with b - a <= h every window
//     (i-o, i+u] contains row c = a + u, so its extremum is ext(suffix
//     extremum of rows i-o+1 .. c, prefix extremum of rows c+1 .. i+u).  One
//     backward sweep of h rows stores the suffixes, one forward sweep of
//     b - a - 1 rows combines them with the running prefix.  Four columns
//     are packed per 32-bit word (byte-wise vmin/vmax).
//  2. horizontal: on each row of vertical extrema (in shared memory) the
//     extremum over 2^k consecutive columns is built by K = floor(log2 w)
//     doubling steps, and the window's extremum is ext(M_K[start],
//     M_K[start + w - 2^K]) (two overlapping blocks cover the window).
// Pixels outside the image take no part: they read as 0xFF for the minimum
// and 0x00 for the maximum.
#include "bz_internal.h"

namespace bz {

constexpr int kMmThreads = 128;            // 4 warps
constexpr int kMmTileCols = 512;           // TW
constexpr int kMmTileRows = 32;            // TR
constexpr int kMmMaxWords = 3;             // vertical words per thread (NWd <= 384)
constexpr int kMmBatch = 8;                // rows loaded together in the vertical sweeps

enum MmOut : int { MM_EXTREMA = 0, MM_BERNSEN = 1 };

// Words of one extended row: 4 columns each, from xa = floor4(x0 - (l-1))
// through x0 + TW - 1 + r, plus 34 words of padding for the shifted reads.
__host__ __device__ inline int mm_words(int w)
{
    return (kMmTileCols + w - 1 + 3) / 4 + 1;
}
__host__ __device__ inline int mm_pitch_words(int w)
{
    return mm_words(w) + 34;
}

template <bool VEC4>
__device__ __forceinline__ uint32_t mm_load(const Image &g, int64_t row, int64_t xw)
{
    const uint8_t *rp = g.img + row * g.pitch;
    if (VEC4 && xw >= 0 && xw + 4 <= g.W)
        return BZ_DBG_IN(rp + xw, 4, g.img, dbg_image_extent(g), kDbgImage)
                   ? __ldg(reinterpret_cast<const uint32_t *>(rp + xw))
                   : 0u;
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int64_t c = xw + b;
        if (c >= 0 && c < g.W)
            v |= (uint32_t)rp[c] << (8 * b);
    }
    return v;
}

// 16-bit pair minimum / maximum (one instruction; the byte-quad __vminu4 /
// __vmaxu4 take several).  The vertical sweeps keep a word's 4 columns as two
// pairs: columns 0, 1 (lo) and 2, 3 (hi), each byte widened to 16 bits.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t pair_lo(uint32_t w)
{
    return __byte_perm(w, 0u, 0x4140u);
}
__device__ __forceinline__ uint32_t pair_hi(uint32_t w)
{
    return __byte_perm(w, 0u, 0x4342u);
}
__device__ __forceinline__ uint32_t pairs_pack(uint32_t lo, uint32_t hi)
{
    return __byte_perm(lo, hi, 0x6420u);
}

// Bytes [byte, byte+4) of a shared-memory row of words.
__device__ __forceinline__ uint32_t mm_bytes(const uint32_t *row, int byte)
{
    const int q = byte >> 2, s = byte & 3;
    return __funnelshift_r(row[q], row[q + 1], 8 * s);
}

template <int OUT, bool VEC4>
__global__ void __launch_bounds__(kMmThreads)
    k_minmax(Image g, Window win, int32_t contrast_limit, uint8_t *mn_out, uint8_t *mx_out,
             uint8_t *bits, int64_t out_pitch, int64_t tiles_x)
{
    extern __shared__ uint32_t mm_smem[];
    const int NWd = mm_words(win.w), NWP = mm_pitch_words(win.w);
    uint32_t *Vmin = mm_smem;                        // [TR][NWP]
    uint32_t *Vmax = mm_smem + kMmTileRows * NWP;    // [TR][NWP]
    // per-warp scratch rows for the doubling steps (ping-pong with the row)
    uint32_t *Smin = mm_smem + 2 * kMmTileRows * NWP + (threadIdx.x >> 5) * NWP;
    uint32_t *Smax = Smin + (kMmThreads / 32) * NWP;

    const int64_t tx = (int64_t)blockIdx.x % tiles_x, ty = (int64_t)blockIdx.x / tiles_x;
    const int64_t x0 = tx * kMmTileCols, y0 = ty * kMmTileRows;
    const int64_t y1 = y0 + kMmTileRows < g.H ? y0 + kMmTileRows : g.H;
    const int l = win.l, o = win.o, u = win.u, h = win.h, w = win.w;
    const int64_t xs = x0 - (l - 1);
    const int64_t xa = xs >= 0 ? (xs & ~(int64_t)3) : -((-xs + 3) & ~(int64_t)3);
    const int delta = (int)(xs - xa);
    const int tid = threadIdx.x;

    // padding words: neutral
    for (int q = NWd + tid; q < NWP; q += kMmThreads)
        for (int i = 0; i < kMmTileRows; i++) {
            Vmin[i * NWP + q] = 0xFFFFFFFFu;
            Vmax[i * NWP + q] = 0u;
        }
    for (int q = NWd + (threadIdx.x & 31); q < NWP; q += 32) {
        Smin[q] = 0xFFFFFFFFu;
        Smax[q] = 0u;
    }

    // ---- 1. vertical extrema, per word column ----
    uint32_t oob[kMmMaxWords];
    int64_t xw[kMmMaxWords];
    bool act[kMmMaxWords];
#pragma unroll
    for (int m = 0; m < kMmMaxWords; m++) {
        const int q = tid + m * kMmThreads;
        act[m] = q < NWd;
        xw[m] = xa + 4 * (int64_t)q;
        uint32_t mk = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int64_t c = xw[m] + b;
            if (c < 0 || c >= g.W)
                mk |= 0xFFu << (8 * b);
        }
        oob[m] = mk;
    }
    uint32_t oobl[kMmMaxWords], oobh[kMmMaxWords];  // the masks as pairs (0x00FF: outside)
#pragma unroll
    for (int m = 0; m < kMmMaxWords; m++) {
        oobl[m] = pair_lo(oob[m]);
        oobh[m] = pair_hi(oob[m]);
    }
    for (int64_t a = y0; a < y1; a += h) {
        const int64_t b = a + h < y1 ? a + h : y1;
        const int64_t c = a + u;
        // backward sweep: suffix extrema of rows s .. c, stored for the
        // window starts s = i-o+1, i in [a, b)
        uint32_t sminl[kMmMaxWords], sminh[kMmMaxWords], smaxl[kMmMaxWords], smaxh[kMmMaxWords];
#pragma unroll
        for (int m = 0; m < kMmMaxWords; m++) {
            sminl[m] = sminh[m] = 0x00FF00FFu;
            smaxl[m] = smaxh[m] = 0u;
        }
        // (rows are loaded kMmBatch at a time so that their latencies overlap)
        for (int64_t s0 = c; s0 >= a - o + 1; s0 -= kMmBatch) {
            uint32_t v[kMmBatch][kMmMaxWords];
#pragma unroll
            for (int k = 0; k < kMmBatch; k++) {
                const int64_t s = s0 - k;
                const bool in = s >= a - o + 1 && s >= 0 && s < g.H;
#pragma unroll
                for (int m = 0; m < kMmMaxWords; m++)
                    v[k][m] = (in && act[m]) ? mm_load<VEC4>(g, s, xw[m]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kMmBatch; k++) {
                const int64_t s = s0 - k;
                if (s < a - o + 1)
                    break;
                if (s >= 0 && s < g.H) {
#pragma unroll
                    for (int m = 0; m < kMmMaxWords; m++) {
                        const uint32_t vl = pair_lo(v[k][m]), vh = pair_hi(v[k][m]);
                        sminl[m] = min_u16x2(sminl[m], vl | oobl[m]);
                        sminh[m] = min_u16x2(sminh[m], vh | oobh[m]);
                        smaxl[m] = max_u16x2(smaxl[m], vl & ~oobl[m]);
                        smaxh[m] = max_u16x2(smaxh[m], vh & ~oobh[m]);
                    }
                }
                const int64_t i = s + o - 1;  // the output row whose window starts at s
                if (i >= a && i < b) {
#pragma unroll
                    for (int m = 0; m < kMmMaxWords; m++) {
                        if (act[m]) {
                            const int q = tid + m * kMmThreads;
                            Vmin[(i - y0) * NWP + q] = pairs_pack(sminl[m], sminh[m]);
                            Vmax[(i - y0) * NWP + q] = pairs_pack(smaxl[m], smaxh[m]);
                        }
                    }
                }
            }
        }
        // forward sweep: prefix extrema of rows c+1 .. i+u
        uint32_t pminl[kMmMaxWords], pminh[kMmMaxWords], pmaxl[kMmMaxWords], pmaxh[kMmMaxWords];
#pragma unroll
        for (int m = 0; m < kMmMaxWords; m++) {
            pminl[m] = pminh[m] = 0x00FF00FFu;
            pmaxl[m] = pmaxh[m] = 0u;
        }
        for (int64_t i0 = a + 1; i0 < b; i0 += kMmBatch) {
            uint32_t v[kMmBatch][kMmMaxWords];
#pragma unroll
            for (int k = 0; k < kMmBatch; k++) {
                const int64_t q_row = i0 + k + u;
                const bool in = i0 + k < b && q_row < g.H;
#pragma unroll
                for (int m = 0; m < kMmMaxWords; m++)
                    v[k][m] = (in && act[m]) ? mm_load<VEC4>(g, q_row, xw[m]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kMmBatch; k++) {
                const int64_t i = i0 + k;
                if (i >= b)
                    break;
#pragma unroll
                for (int m = 0; m < kMmMaxWords; m++) {
                    if (act[m]) {
                        if (i + u < g.H) {
                            const uint32_t vl = pair_lo(v[k][m]), vh = pair_hi(v[k][m]);
                            pminl[m] = min_u16x2(pminl[m], vl | oobl[m]);
                            pminh[m] = min_u16x2(pminh[m], vh | oobh[m]);
                            pmaxl[m] = max_u16x2(pmaxl[m], vl & ~oobl[m]);
                            pmaxh[m] = max_u16x2(pmaxh[m], vh & ~oobh[m]);
                        }
                        const int q = tid + m * kMmThreads;
                        const int64_t x = (i - y0) * NWP + q;
                        const uint32_t a = Vmin[x], b = Vmax[x];
                        Vmin[x] = pairs_pack(min_u16x2(pair_lo(a), pminl[m]), min_u16x2(pair_hi(a), pminh[m]));
                        Vmax[x] = pairs_pack(max_u16x2(pair_lo(b), pmaxl[m]), max_u16x2(pair_hi(b), pmaxh[m]));
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---- 2. horizontal extrema by doubling, one warp per row ----
    const int warp = tid >> 5, lane = tid & 31;
    int K = 0;
    while ((2 << K) <= w)
        K++;
    const int rows = (int)(y1 - y0);
    for (int i = warp; i < rows; i += kMmThreads / 32) {
        uint32_t *rmin = Vmin + i * NWP, *rmax = Vmax + i * NWP;
        uint32_t *tmin = Smin, *tmax = Smax;
        for (int k = 1; k <= K; k++) {
            const int sh = 1 << (k - 1);  // bytes
            for (int q = lane; q < NWd; q += 32) {
                tmin[q] = __vminu4(rmin[q], mm_bytes(rmin, 4 * q + sh));
                tmax[q] = __vmaxu4(rmax[q], mm_bytes(rmax, 4 * q + sh));
            }
            __syncwarp();
            uint32_t *x = rmin;  // the new extrema become the current row
            rmin = tmin;
            tmin = x;
            x = rmax;
            rmax = tmax;
            tmax = x;
        }
        // window extremum of output column x0 + 4p + e: bytes at start
        // 4p + delta and 4p + delta + w - 2^K
        const int64_t row = y0 + i;
        const int second = w - (1 << K);
        if (OUT == MM_EXTREMA) {
            for (int p = lane; p < kMmTileCols / 4; p += 32) {
                const int64_t j0 = x0 + 4 * p;
                if (j0 >= g.W)
                    break;
                const uint32_t lo = __vminu4(mm_bytes(rmin, 4 * p + delta),
                                             mm_bytes(rmin, 4 * p + delta + second));
                const uint32_t hi = __vmaxu4(mm_bytes(rmax, 4 * p + delta),
                                             mm_bytes(rmax, 4 * p + delta + second));
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    if (j0 + e < g.W && BZ_DBG_IN(mn_out + row * g.W + j0 + e, 1, mn_out, (size_t)(g.H * g.W), kDbgOutput) &&
                        BZ_DBG_IN(mx_out + row * g.W + j0 + e, 1, mx_out, (size_t)(g.H * g.W), kDbgOutput)) {
                        mn_out[row * g.W + j0 + e] = (uint8_t)(lo >> (8 * e));
                        mx_out[row * g.W + j0 + e] = (uint8_t)(hi >> (8 * e));
                    }
                }
            }
        } else {
            for (int p = lane; p < kMmTileCols / 8; p += 32) {
                const int64_t j0 = x0 + 8 * p;
                if (j0 >= g.W)
                    break;
                uint32_t byte = 0;
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    const int pw = 2 * p + half;
                    const uint32_t lo = __vminu4(mm_bytes(rmin, 4 * pw + delta),
                                                 mm_bytes(rmin, 4 * pw + delta + second));
                    const uint32_t hi = __vmaxu4(mm_bytes(rmax, 4 * pw + delta),
                                                 mm_bytes(rmax, 4 * pw + delta + second));
                    const uint32_t I4 = mm_load<VEC4>(g, row, j0 + 4 * half);
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int32_t I = (int32_t)((I4 >> (8 * e)) & 0xFFu);
                        const int32_t mn = (int32_t)((lo >> (8 * e)) & 0xFFu);
                        const int32_t mx = (int32_t)((hi >> (8 * e)) & 0xFFu);
                        const uint32_t bit = (mx - mn >= contrast_limit) ? (2 * I > mn + mx)
                                                                          : (mn + mx > 255);
                        byte |= bit << (4 * half + e);
                    }
                }
                if (j0 + 8 > g.W)
                    byte &= (1u << (g.W - j0)) - 1u;  // padding bits are 0
                if (BZ_DBG_IN(bits + row * out_pitch + (j0 >> 3), 1, bits,
                              dbg_extent(g.H, out_pitch, (g.W + 7) / 8), kDbgOutput))
                    bits[row * out_pitch + (j0 >> 3)] = (uint8_t)byte;
            }
        }
        __syncwarp();  // the scratch rows are rewritten by the next row
    }
}

template <int OUT, bool VEC4>
static cudaError_t launch_mm_t(const Image &g, const Window &win, int32_t contrast_limit,
                               uint8_t *mn, uint8_t *mx, uint8_t *bits, int64_t out_pitch,
                               cudaStream_t stream)
{
    // the shared-memory opt-in (largest window), once per device
    static unsigned long long configured = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const size_t smem =
        (size_t)(2 * kMmTileRows + 2 * (kMmThreads / 32)) * mm_pitch_words(511) * sizeof(uint32_t);
    if (dev >= 64 || !(configured >> dev & 1ull)) {
        e = cudaFuncSetAttribute(k_minmax<OUT, VEC4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess)
            return e;
        if (dev < 64)
            configured |= 1ull << dev;
    }
    const size_t need =
        (size_t)(2 * kMmTileRows + 2 * (kMmThreads / 32)) * mm_pitch_words(win.w) * sizeof(uint32_t);
    const int64_t tiles_x = (g.W + kMmTileCols - 1) / kMmTileCols;
    const int64_t tiles = tiles_x * ((g.H + kMmTileRows - 1) / kMmTileRows);
    if (tiles > 2147483647LL)
        return cudaErrorInvalidValue;
    k_minmax<OUT, VEC4><<<(unsigned)tiles, kMmThreads, need, stream>>>(g, win, contrast_limit, mn, mx,
                                                                       bits, out_pitch, tiles_x);
    return cudaGetLastError();
}

cudaError_t launch_minmax(const Image &g, const Window &win, int32_t contrast_limit, uint8_t *mn,
                          uint8_t *mx, uint8_t *bits, int64_t out_pitch, cudaStream_t stream)
{
    const bool vec4 = ((uintptr_t)g.img % 4 == 0) && (g.pitch % 4 == 0);
    if (bits)
        return vec4 ? launch_mm_t<MM_BERNSEN, true>(g, win, contrast_limit, mn, mx, bits, out_pitch, stream)
                    : launch_mm_t<MM_BERNSEN, false>(g, win, contrast_limit, mn, mx, bits, out_pitch,
                                                     stream);
    return vec4 ? launch_mm_t<MM_EXTREMA, true>(g, win, contrast_limit, mn, mx, bits, out_pitch, stream)
                : launch_mm_t<MM_EXTREMA, false>(g, win, contrast_limit, mn, mx, bits, out_pitch, stream);
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_minmax)

}  // namespace bz
