// Local-quantile kernel: one block per (column strip, row band) tile.
#include "bz_internal.h"
#include "bz_quantile.cuh"

namespace bz {

template <typename CT, int NT>
__global__ void __launch_bounds__(NT)
    k_quantile(Image g, Window win, int32_t q_num, int32_t q_den, int32_t offset, uint8_t *out,
               int64_t out_pitch, uint8_t *Qout, int64_t tiles_x, int64_t tile_h)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int64_t x0 = tx * NT, y0 = ty * tile_h;
    const int64_t y1 = y0 + tile_h < g.H ? y0 + tile_h : g.H;
    quantile_tile<CT, NT>(g, win, q_num, q_den, offset, out, out_pitch, Qout, x0, y0, y1, smem);
}

template <typename CT, int NT>
static cudaError_t launch_q(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream)
{
    const size_t smem = quantile_smem_bytes<NT>(sizeof(CT), win.w);
    cudaError_t e = cudaFuncSetAttribute(k_quantile<CT, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    // One wave: as many row bands as the resident-block slots allow for the
    // column strips (the histograms in shared memory cap residency at a few
    // blocks per SM, so a second, partial wave would leave most SMs idle).
    int dev = 0, sms = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_quantile<CT, NT>, NT, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t tiles_x = (g.W + NT - 1) / NT;
    int64_t bands = ((int64_t)sms * per_sm) / tiles_x;
    if (bands < 1)
        bands = 1;
    int64_t tile_h = (g.H + bands - 1) / bands;
    if (tile_h < 1)
        tile_h = 1;
    const int64_t tiles_y = (g.H + tile_h - 1) / tile_h;
    k_quantile<CT, NT><<<(unsigned)(tiles_x * tiles_y), NT, smem, stream>>>(
        g, win, q_num, q_den, offset, out, out_pitch, Q, tiles_x, tile_h);
    return cudaGetLastError();
}

cudaError_t launch_quantile(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream)
{
    if ((int64_t)win.h * win.w <= 65535)
        return launch_q<uint16_t, 128>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
    return launch_q<uint32_t, 64>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
}

}  // namespace bz
