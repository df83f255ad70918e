// Batched execution: many images of uneven sizes and windows in one launch.
//
// The host turns the jobs into a device work list (a header plus one
// descriptor per job with the first global tile index of the job) and runs a
// CUDA graph [H2D copy of the list -> reset of the FP64-fallback counter ->
// persistent window kernel -> persistent quantile kernel] on the caller's
// stream.  Persistent warps (window path) and blocks (quantile path) pop
// global tile indices from atomic counters in the list header, find the job
// by binary search over the tile offsets, and run the same tile routines as
// the single-image kernels, so every result is bit-identical to the
// single-image call.  The graph topology is fixed per precision; only the
// list contents change between launches.
#include <stddef.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "batch_internal.h"
#include "bz_quantile.cuh"

namespace bz {

constexpr int kBatchWarps = 4;   // warps per block, window kernel

// Window tiles of kernel class CLS (see BatchHeader): tiles popped from the
// class's cursor, the job found by binary search over its segment.
template <int MODE, int CLS>
__global__ void __launch_bounds__(32 * kBatchWarps, CLS < 2 ? kBlocksPerSM : 1)
    k_batch_window(BatchHeader *hdr, const WinJobDev *jobs_all, unsigned long long *fallbacks)
{
    constexpr bool kPipe = CLS < 2 && (MODE == MODE_FP64 || MODE == MODE_FP32);
    __shared__ uint4 slots[kBatchWarps][kPipe ? kPipeSlots : 1];  // pipelined path
    const int lane = threadIdx.x & 31;
    const WinJobDev *jobs = jobs_all + hdr->cls_begin[CLS];
    const int64_t total = hdr->cls_tiles[CLS];
    const int nj = hdr->cls_n[CLS];
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0)
            t = atomicAdd(&hdr->cls_next[CLS], 1ull);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if ((int64_t)t >= total)
            break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].tile_begin <= (int64_t)t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const WinJobDev &J = jobs[lo];
        const int64_t local = (int64_t)t - J.tile_begin;
        const int64_t tx = local % J.tiles_x, ty = local / J.tiles_x;
        const int64_t x0 = tx * kTileCols, y0 = ty * J.tile_h;
        const int64_t y1 = y0 + J.tile_h < J.g.H ? y0 + J.tile_h : J.g.H;
        Outputs o{};
        o.bits = J.out;
        o.out_pitch = J.out_pitch;
        o.bits_bytes = dbg_extent(J.g.H, J.out_pitch, (J.g.W + 7) / 8);
        o.fallbacks = fallbacks;
        if (kPipe) {
            window_tile<MODE, true, uint32_t, kPipe ? CLS + 1 : 0>(J.g, J.win, J.T, o, x0, y0, y1, lane,
                                                                   slots[threadIdx.x >> 5]);
        } else if (J.vec) {
            if (J.wide)
                window_tile<MODE, true, unsigned long long, 0>(J.g, J.win, J.T, o, x0, y0, y1, lane,
                                                            nullptr);
            else
                window_tile<MODE, true, uint32_t, 0>(J.g, J.win, J.T, o, x0, y0, y1, lane, nullptr);
        } else {
            if (J.wide)
                window_tile<MODE, false, unsigned long long, 0>(J.g, J.win, J.T, o, x0, y0, y1, lane,
                                                             nullptr);
            else
                window_tile<MODE, false, uint32_t, 0>(J.g, J.win, J.T, o, x0, y0, y1, lane, nullptr);
        }
    }
}

// One warp per block; each warp pops quantile tiles (32 columns x a row band)
// and runs the single-image tile routine in its own shared-memory arrays.
__global__ void __launch_bounds__(32) k_batch_quantile(BatchHeader *hdr, const QJobDev *jobs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    QWarpSmem &S = *reinterpret_cast<QWarpSmem *>(smem);
    const int lane = threadIdx.x & 31;
    const int64_t total = hdr->q_tiles;
    const int nj = hdr->n_q;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0)
            t = atomicAdd(&hdr->q_next, 1ull);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if ((int64_t)t >= total)
            break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].tile_begin <= (int64_t)t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const QJobDev &J = jobs[lo];
        const int64_t local = (int64_t)t - J.tile_begin;
        const int64_t tx = local % J.tiles_x, ty = local / J.tiles_x;
        const int64_t x0 = tx * kQCols, y0 = ty * J.tile_h;
        const int64_t y1 = y0 + J.tile_h < J.g.H ? y0 + J.tile_h : J.g.H;
        // the batch takes the generic read-ahead width (one instantiation
        // keeps the persistent kernel small); results do not depend on it
        if (J.win.w >= 32)
            quantile_warp_tile<6, true>(J.g, J.win, J.q_num, J.q_den, J.offset, J.out, J.out_pitch,
                                        nullptr, x0, y0, y1, S, lane);
        else
            quantile_warp_tile<2, false>(J.g, J.win, J.q_num, J.q_den, J.offset, J.out, J.out_pitch,
                                         nullptr, x0, y0, y1, S, lane);
    }
}

static size_t batch_quant_smem() { return sizeof(QWarpSmem); }

// ------------------------------------------------------------------ host --
bz_status validate_job(const bz_job &j)
{
    bz_status st = check_image(j.image, j.H, j.W, j.in_pitch, j.h, j.w);
    if (st != BZ_OK)
        return st;
    st = check_out(j.image, j.H, j.W, j.in_pitch, j.out, j.out_pitch);
    if (st != BZ_OK)
        return st;
    if (j.method == BZ_QUANTILE) {
        if (j.q_den < 1 || j.q_num < 0 || j.q_num > j.q_den || j.offset < -255 || j.offset > 255)
            return BZ_EINVAL;
    } else if (j.method == BZ_SAUVOLA || j.method == BZ_NIBLACK) {
        if (!isfinite(j.k) || fabs(j.k) > 1e6)
            return BZ_EINVAL;
        if (j.method == BZ_SAUVOLA && (!isfinite(j.R) || j.R < 1e-6 || j.R > 1e9))
            return BZ_EINVAL;
    } else {
        return BZ_EINVAL;
    }
    return BZ_OK;
}

// Tile rows of a batched job: `mult` window heights (in a batch the
// parallelism comes from many images, so tiles are tall), at least 48 rows
// (window jobs) or 64 (quantile jobs).  The multipliers are 3 and 2 unless
// the autotuner's cache holds others for this GPU and precision.
constexpr int kBatchWinMult = 3, kBatchQuantMult = 2;

static int64_t batch_tile_rows(int64_t H, int h, int mult = kBatchWinMult)
{
    int64_t th = (int64_t)mult * h;
    if (th < 48)
        th = 48;
    if (th > H)
        th = H;
    return th;
}

static int64_t quant_tile_rows(int64_t H, int h, int mult = kBatchQuantMult)
{
    int64_t th = (int64_t)mult * h;
    if (th < 64)
        th = 64;
    if (th > H)
        th = H;
    return th;
}

static int batch_mode_of(int precision_mode)
{
    return precision_mode == 0 ? MODE_FP64 : (precision_mode == 1 ? MODE_FP32 : MODE_FP64_DIRECT);
}

// Kernel class of a window job (see BatchHeader).
static int window_class(const bz_job &j, int precision_mode)
{
    const bool vec = ((uintptr_t)j.image % 8 == 0) && (j.in_pitch % 8 == 0);
    const bool s2_32 = (int64_t)j.h * j.w <= 66051;
    const int aw = pipe_words(batch_mode_of(precision_mode), vec, s2_32, Image{j.image, j.H, j.W, j.in_pitch},
                              make_window(j.h, j.w));
    return aw == 1 ? 0 : (aw == 2 ? 1 : 2);
}

// The window jobs order[0 .. n) of `jobs` into `out`: grouped by kernel
// class, most expensive tiles (longest warm-up + tile) first within a class,
// with tile rows mult * h (batch_tile_rows); fills the header's class
// fields.  Reorders `order`; allocates nothing.
static void fill_window_jobs(const bz_job *jobs, int *order, int n, int precision_mode, int mult,
                             WinJobDev *out, BatchHeader *hdr)
{
    std::sort(order, order + n, [&](int a, int b) {
        const int ca = window_class(jobs[a], precision_mode), cb = window_class(jobs[b], precision_mode);
        if (ca != cb)
            return ca < cb;
        const int64_t wa = batch_tile_rows(jobs[a].H, jobs[a].h, mult) + jobs[a].h;
        const int64_t wb = batch_tile_rows(jobs[b].H, jobs[b].h, mult) + jobs[b].h;
        return wa != wb ? wa > wb : a < b;
    });
    for (int c = 0; c < kWinClasses; c++) {
        hdr->cls_begin[c] = 0;
        hdr->cls_n[c] = 0;
        hdr->cls_tiles[c] = 0;
        hdr->cls_next[c] = 0;
    }
    int c_prev = -1;
    int64_t tb = 0;
    for (int a = 0; a < n; a++) {
        const bz_job &j = jobs[order[a]];
        const int c = window_class(j, precision_mode);
        if (c != c_prev) {
            hdr->cls_begin[c] = a;
            tb = 0;
            c_prev = c;
        }
        WinJobDev &d = out[a];
        d.g = Image{j.image, j.H, j.W, j.in_pitch};
        d.win = make_window(j.h, j.w);
        d.T = make_thresh(j.method == BZ_SAUVOLA ? 0 : 1, j.k, j.method == BZ_SAUVOLA ? j.R : 128.0);
        d.out = j.out;
        d.out_pitch = j.out_pitch;
        d.tile_h = batch_tile_rows(j.H, j.h, mult);
        d.tiles_x = (j.W + kTileCols - 1) / kTileCols;
        d.tile_begin = tb;
        d.vec = ((uintptr_t)j.image % 8 == 0) && (j.in_pitch % 8 == 0);
        d.wide = (int64_t)j.h * j.w > 66051;
        tb += d.tiles_x * ((j.H + d.tile_h - 1) / d.tile_h);
        hdr->cls_n[c]++;
        hdr->cls_tiles[c] = tb;
    }
}

// Grids of the persistent kernels: SMs x resident blocks of each.
template <int MODE>
static void batch_grids(int nsm, size_t qsmem, int grid_w[kWinClasses], int &grid_q)
{
    int occ[kWinClasses] = {0, 0, 0}, occ_q = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_batch_window<MODE, 0>, 32 * kBatchWarps, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_batch_window<MODE, 1>, 32 * kBatchWarps, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_batch_window<MODE, 2>, 32 * kBatchWarps, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_q, k_batch_quantile, 32, qsmem);
    for (int c = 0; c < kWinClasses; c++)
        grid_w[c] = nsm * (occ[c] < 1 ? 1 : occ[c]);
    grid_q = nsm * (occ_q < 1 ? 1 : occ_q);
}

template <int MODE>
static void launch_batch_kernels(BatchHeader *hdr, const WinJobDev *wj, const QJobDev *qj,
                                 unsigned long long *fallbacks, const int grid_w[kWinClasses], int grid_q,
                                 size_t qsmem, cudaStream_t stream)
{
    k_batch_window<MODE, 0><<<grid_w[0], 32 * kBatchWarps, 0, stream>>>(hdr, wj, fallbacks);
    k_batch_window<MODE, 1><<<grid_w[1], 32 * kBatchWarps, 0, stream>>>(hdr, wj, fallbacks);
    k_batch_window<MODE, 2><<<grid_w[2], 32 * kBatchWarps, 0, stream>>>(hdr, wj, fallbacks);
    k_batch_quantile<<<grid_q, 32, qsmem, stream>>>(hdr, qj);
}

BatchSlot::~BatchSlot()
{
    release();
}

void BatchSlot::release()
{
    for (int m = 0; m < 3; m++)
        if (exec[m]) {
            cudaGraphExecDestroy(exec[m]);
            exec[m] = nullptr;
        }
    if (d_table)
        cudaFree(d_table);
    if (h_table)
        cudaFreeHost(h_table);
    if (cap_stream)
        cudaStreamDestroy(cap_stream);
    if (done)
        cudaEventDestroy(done);
    d_table = nullptr;
    h_table = nullptr;
    cap_stream = nullptr;
    done = nullptr;
    cap_win = cap_q = 0;
}

static size_t table_bytes(int cap_win, int cap_q)
{
    return sizeof(BatchHeader) + sizeof(WinJobDev) * (size_t)cap_win +
           sizeof(QJobDev) * (size_t)cap_q;
}

static bz_status ensure_capacity(BatchSlot &s, int n_win, int n_q)
{
    if (!s.cap_stream) {
        if (cudaGetDevice(&s.device) != cudaSuccess)
            return BZ_ECUDA;
        if (cudaStreamCreateWithFlags(&s.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return BZ_ECUDA;
        if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess)
            return BZ_ECUDA;
        s.fallbacks = fallback_counter(s.device);
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s.device);
        s.num_sms = nsm > 0 ? nsm : 1;
    }
    if (n_win <= s.cap_win && n_q <= s.cap_q && s.d_table)
        return BZ_OK;
    // grow (power of two) and drop the graphs, which embed the buffer addresses
    int cw = s.cap_win > 0 ? s.cap_win : 64, cq = s.cap_q > 0 ? s.cap_q : 16;
    while (cw < n_win)
        cw *= 2;
    while (cq < n_q)
        cq *= 2;
    if (s.d_table) {
        cudaStreamSynchronize(s.cap_stream);
        cudaEventSynchronize(s.done);
        cudaFree(s.d_table);
        cudaFreeHost(s.h_table);
        s.d_table = nullptr;
        s.h_table = nullptr;
    }
    for (int m = 0; m < 3; m++)
        if (s.exec[m]) {
            cudaGraphExecDestroy(s.exec[m]);
            s.exec[m] = nullptr;
        }
    const size_t bytes = table_bytes(cw, cq);
    if (cudaMalloc(&s.d_table, bytes) != cudaSuccess)
        return BZ_ENOMEM;
    if (cudaMallocHost(&s.h_table, bytes) != cudaSuccess) {
        cudaFree(s.d_table);
        s.d_table = nullptr;
        return BZ_ENOMEM;
    }
    s.cap_win = cw;
    s.cap_q = cq;
    return BZ_OK;
}

template <int MODE>
static cudaError_t capture_graph(BatchSlot &s, cudaGraphExec_t *out)
{
    cudaStream_t cs = s.cap_stream;
    BatchHeader *hdr = (BatchHeader *)s.d_table;
    WinJobDev *wj = (WinJobDev *)(hdr + 1);
    QJobDev *qj = (QJobDev *)(wj + s.cap_win);
    const size_t bytes = table_bytes(s.cap_win, s.cap_q);
    const size_t qsmem = batch_quant_smem();
    cudaError_t e = cudaFuncSetAttribute(k_batch_quantile,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_quantile, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    int grid_w[kWinClasses], grid_q = 0;
    batch_grids<MODE>(s.num_sms, qsmem, grid_w, grid_q);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return e;
    cudaMemcpyAsync(s.d_table, s.h_table, bytes, cudaMemcpyHostToDevice, cs);
    if (s.fallbacks)
        cudaMemsetAsync(s.fallbacks, 0, sizeof(unsigned long long), cs);
    launch_batch_kernels<MODE>(hdr, wj, qj, s.fallbacks, grid_w, grid_q, qsmem, cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess)
        return e;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

bz_status run_batch(BatchSlot &s, const bz_job *jobs, int32_t n, bz_precision precision,
                    cudaStream_t stream)
{
    if (n < 0 || (n > 0 && !jobs))
        return BZ_EINVAL;
    int mode;
    switch (precision) {
    case BZ_FP64: mode = 0; break;
    case BZ_FP32: mode = 1; break;
    case BZ_FP64_DIRECT: mode = 2; break;
    default: return BZ_EINVAL;
    }
    int n_win = 0, n_q = 0;
    for (int32_t i = 0; i < n; i++) {
        const bz_status st = validate_job(jobs[i]);
        if (st != BZ_OK)
            return st;
        if (jobs[i].method == BZ_QUANTILE)
            n_q++;
        else
            n_win++;
    }
    if (n == 0)
        return BZ_OK;
    std::lock_guard<std::mutex> lk(s.mu);
    bz_status st = ensure_capacity(s, n_win, n_q);
    if (st != BZ_OK)
        return st;
    // the previous launch of this slot must have consumed the pinned table
    if (cudaEventSynchronize(s.done) != cudaSuccess)
        return BZ_ECUDA;

    BatchHeader *hdr = (BatchHeader *)s.h_table;
    WinJobDev *wj = (WinJobDev *)(hdr + 1);
    QJobDev *qj = (QJobDev *)(wj + s.cap_win);
    std::vector<int> wi, qi;
    for (int32_t i = 0; i < n; i++)
        (jobs[i].method == BZ_QUANTILE ? qi : wi).push_back(i);
    // the work list for tile multipliers (mw, mq), in the pinned table
    auto fill = [&](int mw, int mq) {
        fill_window_jobs(jobs, wi.data(), (int)wi.size(), mode, mw, wj, hdr);
        // quantile jobs: most expensive tiles first (longest warm-up + tile)
        std::stable_sort(qi.begin(), qi.end(), [&](int a, int b) {
            return (int64_t)jobs[a].w * (quant_tile_rows(jobs[a].H, jobs[a].h, mq) + jobs[a].h) >
                   (int64_t)jobs[b].w * (quant_tile_rows(jobs[b].H, jobs[b].h, mq) + jobs[b].h);
        });
        int64_t tb = 0;
        tb = 0;
        for (size_t a = 0; a < qi.size(); a++) {
            const bz_job &j = jobs[qi[a]];
            QJobDev &d = qj[a];
            d.g = Image{j.image, j.H, j.W, j.in_pitch};
            d.win = make_window(j.h, j.w);
            d.q_num = j.q_num;
            d.q_den = j.q_den;
            d.offset = j.offset;
            d.out = j.out;
            d.out_pitch = j.out_pitch;
            d.tile_h = quant_tile_rows(j.H, j.h, mq);
            d.tiles_x = (j.W + kQCols - 1) / kQCols;
            d.tile_begin = tb;
            tb += d.tiles_x * ((j.H + d.tile_h - 1) / d.tile_h);
        }
        hdr->q_tiles = tb;
        hdr->n_q = n_q;
        hdr->pad0 = 0;
        hdr->q_next = 0;
    };

    const int gi = mode;
    if (!s.exec[gi]) {
        const cudaError_t e = mode == 0   ? capture_graph<MODE_FP64>(s, &s.exec[gi])
                              : mode == 1 ? capture_graph<MODE_FP32>(s, &s.exec[gi])
                                          : capture_graph<MODE_FP64_DIRECT>(s, &s.exec[gi]);
        if (e != cudaSuccess) {
            s.exec[gi] = nullptr;
            cudaGetLastError();
            return BZ_ECUDA;
        }
    }
    auto launch = [&]() -> bz_status {
        if (cudaGraphLaunch(s.exec[gi], stream) != cudaSuccess)
            return BZ_ECUDA;
        if (mode == 0)
            fallback_mark_batch(s.device);
        if (cudaEventRecord(s.done, stream) != cudaSuccess)
            return BZ_ECUDA;
        return BZ_OK;
    };

    // tile multipliers: the cached ones for this GPU and precision, found by
    // a timed search when asked (explicit tuning call or BZ_TUNE=1)
    int mw = kBatchWinMult, mq = kBatchQuantMult;
    if (tune_env() != 0 || tune_forced()) {
        const std::string key = batch_tune_key(mode);
        TuneCfg c;
        bool have = tune_get(key, c);
        if (tune_now(have)) {
            double best = -1.0;
            const int mws[4] = {2, 3, 4, 6}, mqs[4] = {1, 2, 3, 4};
            cudaEvent_t ev0 = nullptr, ev1 = nullptr;
            if (cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess) {
                for (int a = 0; a < 4; a++) {
                    for (int b = 0; b < 4; b++) {
                        float ms = 0.0f, tot = 0.0f;
                        bool ok = true;
                        for (int rep = 0; rep < 3 && ok; rep++) {  // rep 0 untimed
                            ok = cudaEventSynchronize(s.done) == cudaSuccess;
                            fill(mws[a], mqs[b]);
                            ok = ok && cudaEventRecord(ev0, stream) == cudaSuccess && launch() == BZ_OK &&
                                 cudaEventRecord(ev1, stream) == cudaSuccess &&
                                 cudaEventSynchronize(ev1) == cudaSuccess &&
                                 cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess;
                            if (rep > 0)
                                tot += ms;
                        }
                        if (ok && (best < 0.0 || tot / 2.0 < best)) {
                            best = tot / 2.0;
                            c.tile_h = mws[a];
                            c.stripes = mqs[b];
                            c.edge = 1.0f;
                            c.us = (float)(best * 1e3);
                        }
                    }
                }
            }
            if (ev0)
                cudaEventDestroy(ev0);
            if (ev1)
                cudaEventDestroy(ev1);
            cudaGetLastError();
            if (best > 0.0) {
                have = true;
                tune_put(key, c, true);
            }
            if (cudaEventSynchronize(s.done) != cudaSuccess)
                return BZ_ECUDA;
        }
        if (have && c.tile_h >= 1 && c.tile_h <= 16 && c.stripes >= 1 && c.stripes <= 16) {
            mw = c.tile_h;
            mq = c.stripes;
        }
    }
    fill(mw, mq);
    return launch();
}

static BatchSlot *default_slot(int device)
{
    static std::mutex mu;
    static BatchSlot *slots[64] = {nullptr};
    if (device < 0 || device >= 64)
        return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!slots[device])
        slots[device] = new BatchSlot();
    return slots[device];
}

}  // namespace bz

extern "C" bz_status binarize_batch(const bz_job *jobs_host, int32_t n, bz_precision precision,
                                    void *stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return BZ_ECUDA;
    bz::BatchSlot *s = bz::default_slot(dev);
    if (!s)
        return BZ_ECUDA;
    return bz::run_batch(*s, jobs_host, n, precision, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Allocation-free batched entry point.
//
// Some callers cannot allocate device memory when they binarize: services
// that reserve all of the GPU's memory up front in their own arena or caching
// allocator (so a cudaMalloc from inside a library would fail or fragment
// their pool), and latency-critical loops that must never wait on the
// driver's allocator.  binarize_batch keeps its work list in device memory it
// allocates on first use; this variant keeps it in one fixed array that is
// part of the library image instead, so it never allocates.  The cost is a
// hard cap on the number of jobs per call and a single shared work list.
// ---------------------------------------------------------------------------
namespace bz {

constexpr int kNoAllocMaxJobs = BZ_NOALLOC_MAX_JOBS;

struct NoAllocTable {
    BatchHeader hdr;
    unsigned long long fallbacks;  // FP64-fallback counter of the call
    WinJobDev win[kNoAllocMaxJobs];
    QJobDev q[kNoAllocMaxJobs];
};

// The work list of every binarize_batch_noalloc call on a device.  In host
// code this name is only a host-side stand-in: the device address must come
// from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocTable)];

static std::mutex g_noalloc_mu;             // guards the host staging copy
static NoAllocTable g_noalloc_host;         // host staging copy (static storage)
static int g_noalloc_order[kNoAllocMaxJobs];
static void *g_noalloc_dev[64] = {nullptr};  // symbol address per device

// Once per device, with that device current: resolve the device address of
// the static work list.  Returns nullptr on failure.
static void *noalloc_scratch_address(int device)
{
    if (device < 0 || device >= 64)
        return nullptr;
    if (!g_noalloc_dev[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_noalloc_dev[device] = p;
    }
    return g_noalloc_dev[device];
}

// Per device and precision, once: kernel attributes and resident blocks per
// SM of the two persistent kernels (guarded by g_noalloc_mu).
struct NoAllocLaunch {
    bool ready = false;
    int grid_w[kWinClasses] = {0, 0, 0};
    int grid_q = 0;
};
static NoAllocLaunch g_noalloc_launch[64][3];

template <int MODE>
static cudaError_t noalloc_prepare(NoAllocLaunch &L, int nsm)
{
    const size_t qsmem = batch_quant_smem();
    cudaError_t e = cudaFuncSetAttribute(k_batch_quantile,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_quantile, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    batch_grids<MODE>(nsm, qsmem, L.grid_w, L.grid_q);
    L.ready = true;
    return cudaSuccess;
}

template <int MODE>
static cudaError_t noalloc_launch(NoAllocTable *dev, const NoAllocLaunch &L, cudaStream_t stream)
{
    launch_batch_kernels<MODE>(&dev->hdr, dev->win, dev->q, &dev->fallbacks, L.grid_w, L.grid_q,
                               batch_quant_smem(), stream);
    return cudaGetLastError();
}

// Bounds-check status of this file's kernels (debug build; 1 otherwise).
BZ_DEBUG_ACCESSOR(dbg_status_batch)

}  // namespace bz

extern "C" bz_status binarize_batch_noalloc(const bz_job *jobs, int32_t n, bz_precision precision,
                                            void *stream)
{
    using namespace bz;
    if (n < 0 || (n > 0 && !jobs))
        return BZ_EINVAL;
    if (n > kNoAllocMaxJobs)
        return BZ_EINVAL;  // more jobs than the static work list holds
    int mode;
    switch (precision) {
    case BZ_FP64: mode = 0; break;
    case BZ_FP32: mode = 1; break;
    case BZ_FP64_DIRECT: mode = 2; break;
    default: return BZ_EINVAL;
    }
    for (int32_t i = 0; i < n; i++) {
        const bz_status st = validate_job(jobs[i]);
        if (st != BZ_OK)
            return st;
    }
    if (n == 0)
        return BZ_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return BZ_ECUDA;
    if (dev < 0 || dev >= 64)
        return BZ_ECUDA;
    // the static host staging copy is overwritten by the next call, so a
    // captured copy would replay someone else's list
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return BZ_ECUDA;
    }
    if (cap != cudaStreamCaptureStatusNone)
        return BZ_EINVAL;

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocTable *dtab = (NoAllocTable *)noalloc_scratch_address(dev);
    if (!dtab)
        return BZ_ECUDA;
    NoAllocLaunch &L = g_noalloc_launch[dev][mode];
    if (!L.ready) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
            return BZ_ECUDA;
        const cudaError_t pe = mode == 0   ? noalloc_prepare<MODE_FP64>(L, nsm)
                               : mode == 1 ? noalloc_prepare<MODE_FP32>(L, nsm)
                                           : noalloc_prepare<MODE_FP64_DIRECT>(L, nsm);
        if (pe != cudaSuccess) {
            cudaGetLastError();
            return BZ_ECUDA;
        }
    }
    NoAllocTable &t = g_noalloc_host;
    // window jobs by kernel class, most expensive tiles first (as binarize_batch)
    int nw = 0, nq = 0;
    for (int32_t i = 0; i < n; i++)
        if (jobs[i].method != BZ_QUANTILE)
            g_noalloc_order[nw++] = i;
    fill_window_jobs(jobs, g_noalloc_order, nw, mode, kBatchWinMult, t.win, &t.hdr);
    int64_t tb = 0;
    for (int32_t i = 0; i < n; i++)
        if (jobs[i].method == BZ_QUANTILE)
            g_noalloc_order[nq++] = i;
    std::sort(g_noalloc_order, g_noalloc_order + nq, [&](int a, int b) {
        const int64_t ca = (int64_t)jobs[a].w * (quant_tile_rows(jobs[a].H, jobs[a].h) + jobs[a].h);
        const int64_t cb = (int64_t)jobs[b].w * (quant_tile_rows(jobs[b].H, jobs[b].h) + jobs[b].h);
        return ca != cb ? ca > cb : a < b;
    });
    tb = 0;
    for (int a = 0; a < nq; a++) {
        const bz_job &j = jobs[g_noalloc_order[a]];
        QJobDev &d = t.q[a];
        d.g = Image{j.image, j.H, j.W, j.in_pitch};
        d.win = make_window(j.h, j.w);
        d.q_num = j.q_num;
        d.q_den = j.q_den;
        d.offset = j.offset;
        d.out = j.out;
        d.out_pitch = j.out_pitch;
        d.tile_h = quant_tile_rows(j.H, j.h);
        d.tiles_x = (j.W + kQCols - 1) / kQCols;
        d.tile_begin = tb;
        tb += d.tiles_x * ((j.H + d.tile_h - 1) / d.tile_h);
    }
    t.hdr.q_tiles = tb;
    t.hdr.n_q = nq;
    // everything that must start at zero for this call: the two work-list
    // cursors and the fallback counter (the array keeps the previous call's
    // contents otherwise)
    t.hdr.q_next = 0;  // the window cursors were reset by fill_window_jobs
    t.hdr.pad0 = 0;
    t.fallbacks = 0;
    // Only the used part of the list is copied.  The source is pageable host
    // memory: the copy has consumed it when cudaMemcpyAsync returns, so the
    // staging copy may be refilled by the next call.
    const size_t used_win = offsetof(NoAllocTable, win) + sizeof(WinJobDev) * (size_t)nw;
    if (cudaMemcpyAsync(dtab, &t, used_win, cudaMemcpyHostToDevice, (cudaStream_t)stream) !=
        cudaSuccess)
        return BZ_ECUDA;
    if (nq > 0 && cudaMemcpyAsync(dtab->q, t.q, sizeof(QJobDev) * (size_t)nq,
                                  cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
        return BZ_ECUDA;
    const cudaError_t e = mode == 0   ? noalloc_launch<MODE_FP64>(dtab, L, (cudaStream_t)stream)
                          : mode == 1 ? noalloc_launch<MODE_FP32>(dtab, L, (cudaStream_t)stream)
                                      : noalloc_launch<MODE_FP64_DIRECT>(dtab, L, (cudaStream_t)stream);
    return e == cudaSuccess ? BZ_OK : BZ_ECUDA;
}
