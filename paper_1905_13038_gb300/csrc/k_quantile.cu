// Local-quantile kernel: one warp per (32-column strip, row band) tile.
#include <stddef.h>

#include <type_traits>

#include "bz_internal.h"
#include "bz_quantile.cuh"

namespace bz {

template <int NPF, bool CORE, int OB>
__global__ void __launch_bounds__(32)
    k_quantile(Image g, Window win, int32_t q_num, int32_t q_den, int32_t offset, uint8_t *out,
               int64_t out_pitch, uint8_t *Qout, int64_t tiles_x, int64_t tile_h)
{
    extern __shared__ __align__(16) unsigned char smem[];
    typedef QWarpSmemT<quantile_own_words(OB)> Smem;
    Smem &S = *reinterpret_cast<Smem *>(smem);
    const int64_t tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int64_t x0 = tx * kQCols, y0 = ty * tile_h;
    const int64_t y1 = y0 + tile_h < g.H ? y0 + tile_h : g.H;
    quantile_warp_tile<NPF, CORE, OB>(g, win, q_num, q_den, offset, out, out_pitch, Qout, x0, y0, y1, S,
                                       threadIdx.x & 31);
}

template <int NPF, bool CORE, int OB>
static cudaError_t launch_q(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream)
{
    const auto kernel = k_quantile<NPF, CORE, OB>;
    const size_t smem = sizeof(QWarpSmemT<quantile_own_words(OB)>);
    cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    // eight to eleven warps' arrays per SM need the whole shared-memory carve-out
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    const int64_t tiles_x = (g.W + kQCols - 1) / kQCols;
    const TuneCfg *t = tune_override();
    int64_t tile_h = (t && t->tile_h > 0) ? t->tile_h : quantile_band_rows(g.H, g.W, win.h);
    tile_h = tile_h < g.H ? tile_h : g.H;
    const int64_t tiles_y = (g.H + tile_h - 1) / tile_h;
    kernel<<<(unsigned)(tiles_x * tiles_y), 32, smem, stream>>>(g, win, q_num, q_den, offset, out,
                                                                   out_pitch, Q, tiles_x, tile_h);
    return cudaGetLastError();
}

// One wave: as many row bands as the resident warps allow for the column
// strips (the histograms cap residency at a few warps per SM, so a second,
// partial wave would leave most SMs idle).
int64_t quantile_band_rows(int64_t H, int64_t W, int h)
{
    auto occupancy = [](const void *kernel, size_t smem) {
        int v = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, 32, smem) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        return v;
    };
    static int per_sm[3] = {occupancy((const void *)k_quantile<2, false, 8>, sizeof(QWarpSmemT<8>)),
                            occupancy((const void *)k_quantile<2, false, 10>, sizeof(QWarpSmemT<11>)),
                            occupancy((const void *)k_quantile<2, false, 16>, sizeof(QWarpSmemT<16>))};
    const int ob = quantile_own_bits(h);
    const int per = per_sm[ob == 8 ? 0 : (ob == 10 ? 1 : 2)];
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles_x = (W + kQCols - 1) / kQCols;
    int64_t bands = ((int64_t)sms * per) / tiles_x;
    if (bands < 1)
        bands = 1;
    const int64_t tile_h = (H + bands - 1) / bands;
    return tile_h < 1 ? 1 : tile_h;
}

cudaError_t launch_quantile(const Image &g, const Window &win, int32_t q_num, int32_t q_den,
                            int32_t offset, uint8_t *out, int64_t out_pitch, uint8_t *Q,
                            cudaStream_t stream)
{
    const int ob = quantile_own_bits(win.h);
    auto go = [&](auto npf, auto core) -> cudaError_t {
        constexpr int NPF = decltype(npf)::value;
        constexpr bool CORE = decltype(core)::value;
        if (ob == 8)
            return launch_q<NPF, CORE, 8>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
        if (ob == 10)
            return launch_q<NPF, CORE, 10>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
        return launch_q<NPF, CORE, 16>(g, win, q_num, q_den, offset, out, out_pitch, Q, stream);
    };
    auto run = [&]() -> cudaError_t {
        switch (quantile_prefetch(win.w)) {
        case 2:
            return win.w >= 32 ? go(std::integral_constant<int, 2>(), std::true_type())
                               : go(std::integral_constant<int, 2>(), std::false_type());
        case 4: return go(std::integral_constant<int, 4>(), std::true_type());
        default: return go(std::integral_constant<int, 6>(), std::true_type());
        }
    };
    if (tune_env() == 0 && !tune_forced())
        return run();
    const std::string key = quantile_tune_key(q_num, q_den, win, g.H, g.W);
    TuneCfg c;
    bool have = tune_get(key, c);
    if (tune_now(have)) {
        TuneCfg b;
        if (tune_quantile(g, win, run, stream, b)) {
            c = b;
            have = true;
            tune_put(key, c, true);
        }
    }
    TuneScope scope(have ? &c : nullptr);
    return run();
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_quantile)

}  // namespace bz
