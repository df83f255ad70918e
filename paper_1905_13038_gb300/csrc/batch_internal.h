// Batched-execution internals shared by batch.cu and server.cu.
#pragma once
#include <math.h>
#include <mutex>

#include "bz_internal.h"

namespace bz {

// Window jobs go to one of three persistent kernels (kernel classes): 0 and
// 1 the single-image pipelined path with one or two anchor words per lane
// (pipe_words), 2 the generic row routine; each class has its own segment of
// the job array and its own tile cursor, so that each kernel gets its own
// register allocation as the single-image kernels do.
constexpr int kWinClasses = 3;

struct BatchHeader {
    int32_t n_q, pad0;
    int64_t q_tiles;
    unsigned long long q_next;  // work-list cursors (reset by the host copy)
    int32_t cls_begin[kWinClasses], cls_n[kWinClasses];  // job segment of each class
    int64_t cls_tiles[kWinClasses];                       // tiles of each class
    unsigned long long cls_next[kWinClasses];
};

struct WinJobDev {
    Image g;
    Window win;
    Thresh T;
    uint8_t *out;
    int64_t out_pitch;
    int64_t tiles_x, tile_h, tile_begin;
    int32_t vec, wide;
};

struct QJobDev {
    Image g;
    Window win;
    int32_t q_num, q_den, offset;
    uint8_t *out;
    int64_t out_pitch;
    int64_t tiles_x, tile_h, tile_begin;
};

// A reusable launch context: device work list, pinned host staging copy and
// one instantiated graph per precision.  Launches through one slot are
// serialised on its `done` event; independent slots run concurrently.
struct BatchSlot {
    std::mutex mu;
    int device = 0;
    int num_sms = 1;
    int cap_win = 0, cap_q = 0;
    void *d_table = nullptr;
    void *h_table = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t done = nullptr;
    // one graph per precision
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    unsigned long long *fallbacks = nullptr;
    ~BatchSlot();
    void release();
};

bz_status validate_job(const bz_job &j);
bz_status run_batch(BatchSlot &s, const bz_job *jobs, int32_t n, bz_precision precision,
                    cudaStream_t stream);

}  // namespace bz
