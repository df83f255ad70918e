// Local-quantile tile routine (Sec. 3.4: quantiles by recursively maintained
// histograms), shared by the single-image and the batched kernels.
//
// One thread owns one output column and walks down a band of rows with its
// own 256-bin window histogram in shared memory (thread-interleaved layout
// hist[bin][thread], conflict-free).  Moving down one row adds the w pixels
// of row i+u and removes the w pixels of row i-o (the stripe identity of
// Sec. 3.1 applied to histograms; Theta(w) per pixel as the paper states).
// The two rows are staged in shared memory once per block.  The rank-rho
// value Q is tracked incrementally: `below` counts window pixels < Q and Q
// moves up/down until below < rho <= below + hist[Q].
//
// A histogram update is a shared-memory read-modify-write whose next update
// may hit the same bin, so one at a time they form a latency chain.  The
// updates are therefore applied four at a time: the four counters are read
// together, each gets the sum of the deltas of every update in the group
// that names the same bin, and all four are written back (aliased slots
// read the same old value and write the same new one).
#pragma once
#include "bz_window.cuh"

namespace bz {

template <typename CT, int NT>
__device__ __forceinline__ void hist_add4(CT *hist, int tid, int x0, int x1, int x2, int x3, int d0,
                                          int d1, int d2, int d3)
{
    CT *p0 = hist + x0 * NT + tid, *p1 = hist + x1 * NT + tid;
    CT *p2 = hist + x2 * NT + tid, *p3 = hist + x3 * NT + tid;
    const int h0 = *p0, h1 = *p1, h2 = *p2, h3 = *p3;
    const int s0 = d0 + (x1 == x0 ? d1 : 0) + (x2 == x0 ? d2 : 0) + (x3 == x0 ? d3 : 0);
    const int s1 = d1 + (x0 == x1 ? d0 : 0) + (x2 == x1 ? d2 : 0) + (x3 == x1 ? d3 : 0);
    const int s2 = d2 + (x0 == x2 ? d0 : 0) + (x1 == x2 ? d1 : 0) + (x3 == x2 ? d3 : 0);
    const int s3 = d3 + (x0 == x3 ? d0 : 0) + (x1 == x3 ? d1 : 0) + (x2 == x3 ? d2 : 0);
    *p0 = (CT)(h0 + s0);
    *p1 = (CT)(h1 + s1);
    *p2 = (CT)(h2 + s2);
    *p3 = (CT)(h3 + s3);
}

// One block (NT threads) computes output columns [x0, x0+NT) x rows [y0, y1).
// smem: 256*NT counters of type CT followed by two staging rows.
template <typename CT, int NT>
__device__ __forceinline__ void quantile_tile(const Image &g, const Window &win, int32_t q_num,
                                              int32_t q_den, int32_t offset, uint8_t *out,
                                              int64_t out_pitch, uint8_t *Qout, int64_t x0,
                                              int64_t y0, int64_t y1, unsigned char *smem)
{
    CT *hist = reinterpret_cast<CT *>(smem);
    const int ne = NT + win.w - 1;                 // staged columns per row
    const int ne_pad = (ne + 15) & ~15;
    uint8_t *rin = smem + sizeof(CT) * 256 * NT;   // entering row
    uint8_t *rout = rin + ne_pad;                  // leaving row

    const int tid = threadIdx.x;
    const int64_t j = x0 + tid;
    const int l = win.l, r = win.r, oo = win.o, u = win.u;
    const int64_t cstart = x0 - l + 1;  // first staged column

    for (int b = 0; b < 256; b++)
        hist[b * NT + tid] = 0;

    // staged offsets c in [c_lo, c_hi] are this thread's in-image window
    // columns j-l+1+c (out-of-image columns are not counted: clipping rule)
    const int64_t first = j - l + 1;
    const int c_lo = first < 0 ? (int)(-first) : 0;
    const int c_hi = (int)((g.W - 1 - first) < (int64_t)(win.w - 1) ? (g.W - 1 - first)
                                                                    : (int64_t)(win.w - 1));

    auto stage = [&](uint8_t *dst, int64_t row) {
        const bool inrow = row >= 0 && row < g.H;
        const uint8_t *rp = g.img + (inrow ? row : 0) * g.pitch;
        for (int c = tid; c < ne; c += NT) {
            const int64_t col = cstart + c;
            dst[c] = (inrow && col >= 0 && col < g.W) ? rp[col] : (uint8_t)0;
        }
    };

    // warm-up: window rows (y0-o, y0+u]
    for (int64_t a = y0 - oo + 1; a <= y0 + u; a++) {
        if (a < 0 || a >= g.H)
            continue;  // uniform across the block
        __syncthreads();
        stage(rin, a);
        __syncthreads();
        int c = c_lo;
        for (; c + 3 <= c_hi; c += 4)
            hist_add4<CT, NT>(hist, tid, rin[tid + c], rin[tid + c + 1], rin[tid + c + 2],
                              rin[tid + c + 3], 1, 1, 1, 1);
        for (; c <= c_hi; c++)
            hist[(int)rin[tid + c] * NT + tid] += 1;
    }

    const int64_t cols_hi = j + r < g.W - 1 ? j + r : g.W - 1;
    const int64_t cols_lo = j - l > -1 ? j - l : -1;
    const int64_t cols = cols_hi - cols_lo;

    int Q = 0;
    uint32_t below = 0;  // window pixels with value < Q
    const int lane = tid & 31;

    for (int64_t i = y0; i < y1; i++) {
        if (i > y0) {
            const int64_t ra = i + u, rb = i - oo;
            __syncthreads();
            stage(rin, ra);
            stage(rout, rb);
            __syncthreads();
            // entering pixels +1, leaving pixels -1; a row outside the
            // image is staged as zeros and contributes with delta 0
            const int din = ra < g.H ? 1 : 0, dout = rb >= 0 ? -1 : 0;
            int c = c_lo;
            for (; c + 1 <= c_hi; c += 2) {
                const int a0 = rin[tid + c], b0 = rout[tid + c];
                const int a1 = rin[tid + c + 1], b1 = rout[tid + c + 1];
                hist_add4<CT, NT>(hist, tid, a0, b0, a1, b1, din, dout, din, dout);
                below += din * ((a0 < Q) + (a1 < Q)) + dout * ((b0 < Q) + (b1 < Q));
            }
            if (c <= c_hi) {
                const int a0 = rin[tid + c], b0 = rout[tid + c];
                hist[a0 * NT + tid] += din;
                hist[b0 * NT + tid] += dout;
                below += din * (a0 < Q) + dout * (b0 < Q);
            }
        }
        const int64_t rows = (i + u < g.H - 1 ? i + u : g.H - 1) - (i - oo > -1 ? i - oo : -1);
        const int64_t n = rows * (cols > 0 ? cols : 1);
        int64_t rho = (n * (int64_t)q_num + q_den - 1) / q_den;
        if (rho < 1)
            rho = 1;
        if (rho > n)
            rho = n;
        if (j < g.W) {
            // move Q to the rank-rho value
            while (Q < 255 && (int64_t)below + (int64_t)hist[Q * NT + tid] < rho) {
                below += hist[Q * NT + tid];
                Q++;
            }
            while (Q > 0 && (int64_t)below >= rho) {
                Q--;
                below -= hist[Q * NT + tid];
            }
        }
        uint32_t bit = 0;
        if (j < g.W) {
            const int I = g.img[i * g.pitch + j];
            bit = (I <= Q - offset) ? 0u : 1u;
            if (Qout)
                Qout[i * g.W + j] = (uint8_t)Q;
        }
        if (out) {
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
            const int64_t jw = x0 + (tid & ~31);  // first column of this warp
            if (lane < 4) {
                const int64_t c8 = jw + 8 * lane;
                if (c8 < g.W)
                    out[i * out_pitch + (c8 >> 3)] = (uint8_t)(word >> (8 * lane));
            }
        }
    }
}


template <int NT>
__host__ __device__ constexpr size_t quantile_smem_bytes(size_t ct_bytes, int w)
{
    return ct_bytes * 256 * NT + 2 * (size_t)((NT + w - 1 + 15) & ~15);
}

}  // namespace bz
