// Local-quantile kernel: one warp per (32-column strip, row band) tile.
#include <stddef.h>

#include "bz_internal.h"
#include "bz_quantile.cuh"

namespace bz {

template <int NPF, bool CORE>
__global__ void __launch_bounds__(32)
    k_quantile(Image g, Window win, int32_t q_num, int32_t q_den, int32_t offset, uint8_t *out,
               int64_t out_pitch, uint8_t *Qout, int64_t tiles_x, int64_t tile_h)
{
    extern __shared__ __align__(16) unsigned char smem[];
    QWarpSmem &S = *reinterpret_cast<QWarpSmem *>(smem);
    const int64_t tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int64_t x0 = tx * kQCols, y0 = ty * tile_h;
    const int64_t y1 = y0 + tile_h < g.H ? y0 + tile_h : g.H;
    quantile_warp_tile<NPF, CORE>(g, win, q_num, q_den, offset, out, out_pitch, Qout, x0, y0, y1, S,
                       threadIdx.x & 31);
}

template <int NPF, bool CORE>
static cudaError_t launch_q(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream)
{
    const auto kernel = k_quantile<NPF, CORE>;
    const size_t smem = sizeof(QWarpSmem);
    cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    // eight warps' arrays per SM need the whole shared-memory carve-out
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    // One wave: as many row bands as the resident warps allow for the column
    // strips (the histograms cap residency at a few warps per SM, so a
    // second, partial wave would leave most SMs idle).
    int dev = 0, sms = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t tiles_x = (g.W + kQCols - 1) / kQCols;
    int64_t bands = ((int64_t)sms * per_sm) / tiles_x;
    if (bands < 1)
        bands = 1;
    int64_t tile_h = (g.H + bands - 1) / bands;
    if (tile_h < 1)
        tile_h = 1;
    const int64_t tiles_y = (g.H + tile_h - 1) / tile_h;
    kernel<<<(unsigned)(tiles_x * tiles_y), 32, smem, stream>>>(g, win, q_num, q_den, offset, out,
                                                                   out_pitch, Q, tiles_x, tile_h);
    return cudaGetLastError();
}

cudaError_t launch_quantile(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream)
{
    switch (quantile_prefetch(win.w)) {
    case 2:
        return win.w >= 32 ? launch_q<2, true>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream)
                           : launch_q<2, false>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
    case 4: return launch_q<4, true>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
    default: return launch_q<6, true>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
    }
}

}  // namespace bz
