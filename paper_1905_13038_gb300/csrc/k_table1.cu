// Kernels of the other Table 1 methods: the global-statistics reduction
// (L = min I, sum I, sum I^2 over the whole image) and the window kernel
// instantiated with the Wolf / Feng / Rais / NICK / Phansalkar thresholds.
#include <math.h>

#include "bz_internal.h"

namespace bz {

constexpr int kGsThreads = 256;
constexpr int kWarpsPerBlockExt = 4;

// One pass over the image: each thread takes 16-byte chunks of rows
// (grid-stride over H x ceil(W/16) chunks), accumulates the chunk's sum and
// sum of squares with DP4A and its minimum with byte-wise vmin, then the
// block reduces and adds to *gs with one atomic per quantity.
template <bool VEC16>
__device__ __forceinline__ void gs_chunk(const Image &g, int64_t c, int64_t chunks_per_row,
                                         uint32_t (&wd)[4], uint32_t &mn)
{
    const int64_t i = c / chunks_per_row;
    const int64_t j = (c - i * chunks_per_row) * 16;
    const uint8_t *p = g.img + i * g.pitch + j;
    if (VEC16 && j + 16 <= g.W) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        wd[0] = v.x;
        wd[1] = v.y;
        wd[2] = v.z;
        wd[3] = v.w;
        mn = __vminu4(mn, __vminu4(__vminu4(v.x, v.y), __vminu4(v.z, v.w)));
        return;
    }
    uint32_t lo4[4] = {0u, 0u, 0u, 0u}, hi4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int b = 0; b < 16; b++) {
        const bool in = j + b < g.W;
        const uint32_t v = in ? (uint32_t)p[b] : 0u;
        lo4[b >> 2] |= v << (8 * (b & 3));
        hi4[b >> 2] |= (in ? v : 0xFFu) << (8 * (b & 3));  // 0xFF: neutral for min
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        wd[q] = lo4[q];
        mn = __vminu4(mn, hi4[q]);
    }
}

// One pass over the image: each thread takes 16-byte chunks of rows
// (grid-stride over H x ceil(W/16) chunks, four chunks loaded before any is
// summed), accumulates the chunk's sum and sum of squares with DP4A and its
// minimum with byte-wise vmin, then the block reduces and adds to *gs with
// one atomic per quantity.
template <bool VEC16>
__global__ void __launch_bounds__(kGsThreads) k_global_stats(Image g, GStats *gs, int64_t chunks_per_row,
                                                              int64_t chunks)
{
    unsigned long long s1 = 0, s2 = 0;
    uint32_t mn = 0xFFFFFFFFu;  // byte-wise minimum of four lanes of bytes
    const int64_t stride = (int64_t)gridDim.x * kGsThreads;
    for (int64_t c = (int64_t)blockIdx.x * kGsThreads + threadIdx.x; c < chunks; c += 4 * stride) {
        uint32_t wd[4][4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            wd[k][0] = wd[k][1] = wd[k][2] = wd[k][3] = 0u;
            if (c + k * stride < chunks)
                gs_chunk<VEC16>(g, c + k * stride, chunks_per_row, wd[k], mn);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            uint32_t a1 = 0, a2 = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                a1 = __dp4a(wd[k][q], 0x01010101u, a1);
                a2 = __dp4a(wd[k][q], wd[k][q], a2);
            }
            s1 += a1;
            s2 += a2;
        }
    }
    // minimum of the four bytes
    mn = __vminu4(mn, mn >> 16);
    mn = __vminu4(mn, mn >> 8) & 0xFFu;
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, d);
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, d);
    }
    __shared__ unsigned long long sh1[kGsThreads / 32], sh2[kGsThreads / 32];
    __shared__ uint32_t shm[kGsThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh1[warp] = s1;
        sh2[warp] = s2;
        shm[warp] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t1 = 0, t2 = 0;
        uint32_t tm = 0xFFu;
#pragma unroll
        for (int q = 0; q < kGsThreads / 32; q++) {
            t1 += sh1[q];
            t2 += sh2[q];
            tm = shm[q] < tm ? shm[q] : tm;
        }
        atomicMax(&gs->Linv, 255u - tm);
        atomicAdd(&gs->sum, t1);
        atomicAdd(&gs->sumsq, t2);
    }
}

cudaError_t launch_global_stats(const Image &g, GStats *gs, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(gs, 0, sizeof(GStats), stream);
    if (e != cudaSuccess)
        return e;
    const int64_t cpr = (g.W + 15) / 16;
    const int64_t chunks = cpr * g.H;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (chunks + kGsThreads - 1) / kGsThreads;
    const int64_t cap = (int64_t)sms * 8;  // 8 blocks of 256 threads per SM
    if (blocks > cap)
        blocks = cap;
    const bool vec16 = ((uintptr_t)g.img % 16 == 0) && (g.pitch % 16 == 0);
    if (vec16)
        k_global_stats<true><<<(unsigned)blocks, kGsThreads, 0, stream>>>(g, gs, cpr, chunks);
    else
        k_global_stats<false><<<(unsigned)blocks, kGsThreads, 0, stream>>>(g, gs, cpr, chunks);
    return cudaGetLastError();
}

// (L, M, S) and the exact sums of the global-statistics export.
__global__ void k_global_finalize(const GStats *gs, unsigned long long N, double *stats,
                                  uint64_t *sums)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    const GStats G = *gs;
    const Global r = global_lms(G, N);
    stats[0] = r.L;
    stats[1] = r.M;
    stats[2] = r.S;
    if (sums) {
        sums[0] = G.sum;
        sums[1] = G.sumsq;
        sums[2] = N;
    }
}

cudaError_t launch_global_finalize(const GStats *gs, unsigned long long N, double *stats,
                                   uint64_t *sums, cudaStream_t stream)
{
    k_global_finalize<<<1, 32, 0, stream>>>(gs, N, stats, sums);
    return cudaGetLastError();
}

// The window kernel with a Table 1 threshold other than Sauvola/Niblack:
// warp tiles of 256 columns in the window kernel's tile schedule (one wave,
// shorter edge tiles), the general (non-pipelined) row routine on interior
// and edge tiles.
template <int MODE, bool VEC, typename S2T>
__global__ void __launch_bounds__(32 * kWarpsPerBlockExt, 4)
    k_window_ext(Image g, Window win, ThreshExt T, Outputs o, TileSched S, const uint2 *stripes)
{
    fallbacks_clear(o);  // plain launch: ordered after the previous kernel
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * kWarpsPerBlockExt + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlockExt;
    for (int64_t t = wid; t < S.tiles_total; t += stride) {
        int64_t tx, y0, y1;
        const uint2 *st;
        sched_tile(S, g.W, stripes, t, tx, y0, y1, st);
        const int64_t x0 = tx * kTileCols;
        const bool interior = VEC && (x0 - win.l >= 0) && (x0 + kTileCols + win.r <= g.W);
        if (interior)
            window_rows<MODE, VEC, true, S2T, true>(g, win, T, o, x0, y0, y1, lane, st);
        else
            window_rows<MODE, VEC, false, S2T, true>(g, win, T, o, x0, y0, y1, lane, st);
    }
}

// The pipelined window kernel with Table 1 method METHOD (binarize modes,
// launches for which pipe_words gives one anchor word per lane): interior
// and edge tiles both take window_rows_pipe, in the balanced tile schedule.
template <int MODE, int METHOD>
__global__ void __launch_bounds__(32 * kWarpsPerBlockExt, 4)
    k_window_ext_pipe(Image g, Window win, ThreshExt T, Outputs o, TileSched S, const uint2 *stripes)
{
    fallbacks_clear(o);  // plain launch: ordered after the previous kernel
    __shared__ uint4 slots[kWarpsPerBlockExt][kPipeSlots];
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * kWarpsPerBlockExt + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlockExt;
    for (int64_t t = wid; t < S.tiles_total; t += stride) {
        int64_t tx, y0, y1;
        const uint2 *st;
        sched_tile(S, g.W, stripes, t, tx, y0, y1, st);
        const int64_t x0 = tx * kTileCols;
        if ((x0 - win.l >= 0) && (x0 + kTileCols + win.r <= g.W))
            window_rows_pipe<MODE, false, false, 1, METHOD>(g, win, T, o, x0, y0, y1, lane,
                                                            slots[threadIdx.x >> 5], st);
        else
            window_rows_pipe<MODE, false, true, 1, METHOD>(g, win, T, o, x0, y0, y1, lane,
                                                           slots[threadIdx.x >> 5], st);
    }
}

template <int MODE>
static cudaError_t launch_ext_pipe(const Image &g, const Window &win, const ThreshExt &T, const Outputs &o,
                                   cudaStream_t stream)
{
    const int64_t tile_h = window_tile_rows(g.H, g.W, win.h, win.w);
    const int64_t tiles_y = (g.H + tile_h - 1) / tile_h;
    uint2 *stripes = launch_stripes(g, win, 0, tile_h, tiles_y, stream);
    const TileSched S = make_sched(g, win, 0, g.H, true, stripes != nullptr);
    int64_t blocks = (S.tiles_total + kWarpsPerBlockExt - 1) / kWarpsPerBlockExt;
    if (blocks > 2147483647LL)
        blocks = 2147483647LL;
    const dim3 grid((unsigned)blocks), block(32 * kWarpsPerBlockExt);
    switch (T.method) {
    case METHOD_WOLF: k_window_ext_pipe<MODE, METHOD_WOLF><<<grid, block, 0, stream>>>(g, win, T, o, S, stripes); break;
    case METHOD_FENG: k_window_ext_pipe<MODE, METHOD_FENG><<<grid, block, 0, stream>>>(g, win, T, o, S, stripes); break;
    case METHOD_RAIS: k_window_ext_pipe<MODE, METHOD_RAIS><<<grid, block, 0, stream>>>(g, win, T, o, S, stripes); break;
    case METHOD_NICK: k_window_ext_pipe<MODE, METHOD_NICK><<<grid, block, 0, stream>>>(g, win, T, o, S, stripes); break;
    default:
        k_window_ext_pipe<MODE, METHOD_PHANSALKAR><<<grid, block, 0, stream>>>(g, win, T, o, S, stripes);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (stripes && scratch_free(stripes, stream) != cudaSuccess && e == cudaSuccess)
        e = cudaGetLastError();
    return e;
}

template <int MODE, bool VEC, typename S2T>
static cudaError_t launch_ext_t(const Image &g, const Window &win, const ThreshExt &T,
                                const Outputs &o, cudaStream_t stream)
{
    const int64_t tile_h = window_tile_rows(g.H, g.W, win.h, win.w);
    const int64_t tiles_y = (g.H + tile_h - 1) / tile_h;
    uint2 *stripes = launch_stripes(g, win, 0, tile_h, tiles_y, stream);
    const TileSched S = make_sched(g, win, 0, g.H, false, stripes != nullptr);
    int64_t blocks = (S.tiles_total + kWarpsPerBlockExt - 1) / kWarpsPerBlockExt;
    if (blocks > 2147483647LL)
        blocks = 2147483647LL;
    k_window_ext<MODE, VEC, S2T><<<(unsigned)blocks, 32 * kWarpsPerBlockExt, 0, stream>>>(
        g, win, T, o, S, stripes);
    cudaError_t e = cudaGetLastError();
    if (stripes && scratch_free(stripes, stream) != cudaSuccess && e == cudaSuccess)
        e = cudaGetLastError();
    return e;
}

template <int MODE>
static cudaError_t launch_ext_m(const Image &g, const Window &win, const ThreshExt &T,
                                const Outputs &o, cudaStream_t stream)
{
    const bool vec = ((uintptr_t)g.img % 8 == 0) && (g.pitch % 8 == 0);
    const bool wide = (int64_t)win.h * win.w > 66051;
    if ((MODE == MODE_FP64 || MODE == MODE_FP32) && pipe_words(MODE, vec, !wide, g, win) == 1)
        return launch_ext_pipe<MODE == MODE_FP32 ? MODE_FP32 : MODE_FP64>(g, win, T, o, stream);
    if (vec)
        return wide ? launch_ext_t<MODE, true, unsigned long long>(g, win, T, o, stream)
                    : launch_ext_t<MODE, true, uint32_t>(g, win, T, o, stream);
    return wide ? launch_ext_t<MODE, false, unsigned long long>(g, win, T, o, stream)
                : launch_ext_t<MODE, false, uint32_t>(g, win, T, o, stream);
}

cudaError_t launch_window_ext(int mode, const Image &g, const Window &win, const ThreshExt &T,
                              const Outputs &o, cudaStream_t stream)
{
    switch (mode) {
    case MODE_FP64: return launch_ext_m<MODE_FP64>(g, win, T, o, stream);
    case MODE_FP32: return launch_ext_m<MODE_FP32>(g, win, T, o, stream);
    case MODE_FP64_DIRECT: return launch_ext_m<MODE_FP64_DIRECT>(g, win, T, o, stream);
    case MODE_REPORT: return launch_ext_m<MODE_REPORT>(g, win, T, o, stream);
    default: return cudaErrorInvalidValue;
    }
}

// Relative FP32 bound of the Table 1 thresholds: the Sauvola/Niblack bound
// with 2^-40 added for the FP64 formula's own error.
ThreshExt make_thresh_ext(int method, const double *prm, const GStats *gs, unsigned long long N)
{
    ThreshExt T{};
    static_cast<Thresh &>(T) = make_thresh(0, 0.5, 128.0);
    T.method = method;
    T.k = prm[0];
    T.R = prm[1];
    T.X.alpha1 = prm[2];
    T.X.k1 = prm[3];
    T.X.k2 = prm[4];
    T.X.gamma = prm[5];
    T.X.p = prm[6];
    T.X.q = prm[7];
    T.eps = (float)(24.0 / 16777216.0 + 9.094947017729282e-13);  // 24 * 2^-24 + 2^-40
    T.gs = gs;
    T.N = N;
    return T;
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_table1)

}  // namespace bz
