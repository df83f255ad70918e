// Local-quantile tile routine (Sec. 3.4: quantiles from recursively
// maintained histograms), shared by the single-image and the batched kernels.
//
// One warp computes a tile of 32 output columns x a band of rows.  Lane L
// owns output column j = x0 + L and walks down the band; its window holds the
// staged columns [L, L + w - 1] of the span [x0 - l + 1, x0 + 31 + r].  The
// window histogram of a lane is never stored whole: the window's columns are
// split into three parts, each with its own histogram, slid down the rows by
// adding the entering row i + u and removing the leaving row i - o (the
// stripe identity of Sec. 3.1 applied to histograms):
//
//   core   columns [31, w - 1], in every window of the warp      (w - 31 cols)
//   group  columns [8G + 7, 8G + w - 1] minus the core, in every window of
//          the 8-lane group G                                    (<= 24 cols)
//   own    the rest of the lane's window                         (<= 7 cols)
//
// so a row step costs 2 (w - 31) / 32 + 2 * 24 / 8 + 2 * 7 histogram updates
// per lane instead of the 2 w of a private window histogram: the per-pixel
// work no longer grows with w past 31.  Windows narrower than 32 (8) columns
// have no core (no group) part.
//
// The rank-rho value Q of each lane moves incrementally from its value one
// row up: `below` counts the window pixels < Q.  The lane tracks the own part
// of it with every own update; the core and group parts change with updates
// the whole warp or group made, so they are read back after each row from
// the totals of those histograms per 4 gray values (an exclusive prefix of
// which is rebuilt per row) plus at most 3 fine bins.  Then Q moves until
// below < rho <= below + count(Q): one round of loads at Q - 2 .. Q + 1
// settles the usual moves, longer ones take four gray values per round.
//
// Updates are shared-memory atomics without a return value.  The own
// histograms hold 16-bit counts, two lanes per 32-bit word (a lane's counts
// stay below 7 h <= 3577, so no field borrows from or carries into the
// next), 10-bit counts, three lanes per word, for windows of at most 146 rows
// (7 h <= 1022), or 8-bit counts, four lanes per word, for windows of at most
// 36 rows (7 h <= 252): a warp's arrays take 27.5, 22.3 or 19.2 KB, so 8, 10
// or 11 warps share an SM.  Image columns outside [0, W) are staged as the value 256, a bin
// that is counted but never queried, so no update needs a mask.  Each row's
// bytes are loaded one row step ahead into registers, so the global-memory
// latency overlaps the previous row's work.
#pragma once
#include <stddef.h>

#include "bz_window.cuh"

namespace bz {

constexpr int kQCols = 32;         // output columns per warp tile
constexpr int kQSpanCap = 544;     // staged slots per row (span <= 542)
constexpr int kQSentinel = 543;    // a slot that always holds the value 256
constexpr int kQBins = 260;        // gray values 0..255, 256 = outside the image, read-ahead pad
constexpr int kQQuarters = 68;     // totals per 4 gray values: 0..63, 64 = outside the image

// OWNW = 16: 16-bit own counts (lane L in word L >> 1, half L & 1);
// OWNW = 8: 8-bit own counts (lane L in word L >> 2, byte L & 3).
template <int OWNW>
struct QWarpSmemT {
    uint32_t own[kQBins][OWNW];        // own-part counts
    uint32_t core[kQBins];             // core-part histogram
    uint32_t grp[4][kQBins];           // group-part histogram of each 8-lane group
    uint32_t coreQ[4][kQQuarters];     // core totals per 4 gray values, partial per updating group
    uint32_t grpQ[4][kQQuarters];      // group-part totals per 4 gray values
    uint32_t cumCore[kQQuarters];      // core pixels below 4k, k = 0..64
    uint32_t cumGrp[4][kQQuarters];    // group-part pixels below 4k
    uint16_t rin[kQSpanCap];           // staged entering row
    uint16_t rout[kQSpanCap];          // staged leaving row
};
typedef QWarpSmemT<16> QWarpSmem;

// Bits of an own count: a lane's own part holds at most 7 columns x h rows,
// so 8 bits (four lanes per word) serve h <= 36, 10 bits (three lanes per
// word) h <= 146, 16 bits (two lanes per word) every window.
__host__ __device__ constexpr int quantile_own_bits(int h)
{
    return 7 * h <= 255 ? 8 : (7 * h <= 1023 ? 10 : 16);
}
// Own-count words per gray value: 8, 11 or 16.
__host__ __device__ constexpr int quantile_own_words(int bits)
{
    return bits == 8 ? 8 : (bits == 10 ? 11 : 16);
}

// Pixels of a shared part below gray value Q: the prefix up to Q's 4-value
// step plus at most 3 bins.
__device__ __forceinline__ uint32_t q_part_below(const uint32_t *H, const uint32_t *cum, int Q)
{
    const int k = Q >> 2, f = Q & 3;
    const uint4 h = *reinterpret_cast<const uint4 *>(H + 4 * k);
    uint32_t s = cum[k];
    s += f > 0 ? h.x : 0u;
    s += f > 1 ? h.y : 0u;
    s += f > 2 ? h.z : 0u;
    return s;
}

// Prefetched slots per lane for a window w columns wide: 2, 4 or 6 (spans of
// more than 192 columns stage the rest without the read-ahead).
__host__ __device__ constexpr int quantile_prefetch(int w)
{
    return w + 31 <= 64 ? 2 : w + 31 <= 128 ? 4 : 6;
}

// One warp (lane = threadIdx.x & 31) computes output columns [x0, x0 + 32)
// x rows [y0, y1).  out (packed bits) and Qout (dense quantile plane, W per
// row) may each be null.  NPF = quantile_prefetch(w); CORE = (w >= 32);
// OB = quantile_own_bits(h) or more.
template <int NPF, bool CORE, int OB = 16>
__device__ __forceinline__ void quantile_warp_tile(const Image &g, const Window &win, int32_t q_num,
                                                   int32_t q_den, int32_t offset, uint8_t *out,
                                                   int64_t out_pitch, uint8_t *Qout, int64_t x0,
                                                   int64_t y0, int64_t y1,
                                                   QWarpSmemT<quantile_own_words(OB)> &S, int lane)
{
    constexpr int kOW = quantile_own_words(OB);  // words per own-count row
    constexpr int kLPW = OB == 8 ? 4 : (OB == 10 ? 3 : 2);  // lanes per own word
    const int w = win.w, h = win.h;
    const int G = lane >> 3, pos = lane & 7;
    const int64_t span0 = x0 - win.l + 1;  // image column of staged slot 0
    const int span = kQCols - 1 + w;
    const int64_t j = x0 + lane;
    const bool live = j < g.W;
    const int H = (int)g.H;
    [[maybe_unused]] const size_t img_ext = dbg_image_extent(g);

    __syncwarp();  // the previous tile of this warp is done with the arrays
    {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        uint4 *p = reinterpret_cast<uint4 *>(&S);
        constexpr int n16 = (int)(offsetof(QWarpSmemT<kOW>, rin) / 16);
        for (int k = lane; k < n16; k += 32)
            p[k] = z;
        if (lane == 0) {
            S.rin[kQSentinel] = 256;
            S.rout[kQSentinel] = 256;
        }
    }

    // staged slot of each update entry (kQSentinel for entries a window lacks)
    const int nown = w >= 8 ? 7 : w;
    int ok[7];
#pragma unroll
    for (int e = 0; e < 7; e++)
        ok[e] = e < nown ? lane + e + ((w >= 8 && e >= 7 - pos) ? w - 7 : 0) : kQSentinel;
    const int ngrp = w >= 32 ? 24 : (w >= 8 ? w - 7 : 0);
    const int left = 24 - 8 * G;  // group entries left of the core (w >= 32)
    int gk[3];
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const int e = pos + 8 * t;
        gk[t] = e >= ngrp ? kQSentinel : (w >= 32 && e >= left) ? w + e - left : 8 * G + 7 + e;
    }
    uint32_t gmask = 0;  // group entries this lane updates
#pragma unroll
    for (int t = 0; t < 3; t++)
        if (gk[t] != kQSentinel)
            gmask |= 1u << t;
    const int ncore = CORE ? w - 31 : 0;
    const int core_rounds = (ncore + 31) >> 5;
    const bool has_grp = ngrp > 0;
    // own-count step of this lane, its field of an own word, its column
    const int ofield = lane % kLPW;
    const uint32_t dplus = 1u << (OB * ofield);
    const uint32_t dminus = 0u - dplus;
    const uint32_t osel = OB == 8 ? 0x4440u | (unsigned)ofield : (ofield ? 0x4432u : 0x4410u);
    uint32_t *const ownl = &S.own[0][lane / kLPW];
    auto own_count = [&](uint32_t wd) -> uint32_t {
        return OB == 10 ? (wd >> (10 * ofield)) & 0x3FFu : __byte_perm(wd, 0u, osel);
    };

    // prefetched slots lane + 32 t, t < NPF: stored if inside the span,
    // loaded if also inside the image (else the value 256)
    uint32_t smask = 0, lmask = 0;
#pragma unroll
    for (int t = 0; t < NPF; t++) {
        const int k = lane + 32 * t;
        const int64_t col = span0 + k;
        if (k < span) {
            smask |= 1u << t;
            if (col >= 0 && col < g.W)
                lmask |= 1u << t;
        }
    }
    const int64_t lane_off = span0 + lane;  // image column of slot `lane`

    int Q = 0;          // current rank-rho value of this lane
    uint32_t bown = 0;  // own-part pixels below Q

    // Row steps s = 0 .. h - 2 + (y1 - y0): row ra = y0 - o + 1 + s enters,
    // row ra - h leaves (from s = h on); from s = h - 1 on, row
    // i = y0 + s - h + 1 is output after the step.
    const int ra0 = (int)(y0 - win.o + 1);
    const int steps = h - 1 + (int)(y1 - y0);
    uint32_t pin[NPF], pout[NPF];
    int pc = 0;
    auto fetch = [&](int s) {
        const int ra = ra0 + s, rb = ra - h;
        if (ra >= 0 && ra < H) {
            const uint8_t *p = g.img + (int64_t)ra * g.pitch;
#pragma unroll
            for (int t = 0; t < NPF; t++)
                pin[t] = ((lmask >> t & 1u) && BZ_DBG_IN(p + lane_off + 32 * t, 1, g.img, img_ext, kDbgImage))
                             ? (uint32_t)p[lane_off + 32 * t]
                             : 256u;
        }
        if (s >= h && rb >= 0) {
            const uint8_t *p = g.img + (int64_t)rb * g.pitch;
#pragma unroll
            for (int t = 0; t < NPF; t++)
                pout[t] = ((lmask >> t & 1u) && BZ_DBG_IN(p + lane_off + 32 * t, 1, g.img, img_ext, kDbgImage))
                              ? (uint32_t)p[lane_off + 32 * t]
                              : 256u;
        }
        if (s >= h - 1 && live && BZ_DBG_IN(g.img + (y0 + s - h + 1) * g.pitch + j, 1, g.img, img_ext, kDbgImage))
            pc = g.img[(y0 + s - h + 1) * g.pitch + j];
    };
    auto commit = [&](uint16_t *dst, const uint32_t *v, int row) {
#pragma unroll
        for (int t = 0; t < NPF; t++)
            if (smask >> t & 1u)
                dst[lane + 32 * t] = (uint16_t)v[t];
        // slots past the prefetched ones (spans over 192 columns)
        const uint8_t *p = g.img + (int64_t)row * g.pitch;
        for (int k = 32 * NPF + lane; k < span; k += 32) {
            const int64_t col = span0 + k;
            dst[k] = (col >= 0 && col < g.W && BZ_DBG_IN(p + col, 1, g.img, img_ext, kDbgImage)) ? (uint16_t)p[col]
                                                                                           : (uint16_t)256;
        }
    };

    const int64_t cols_hi = j + win.r < g.W - 1 ? j + win.r : g.W - 1;
    const int64_t cols_lo = j - win.l > -1 ? j - win.l : -1;
    const int cols = (int)(cols_hi - cols_lo);
    int rows_prev = -1;
    uint32_t rho = 1;

    if (steps > 0)
        fetch(0);
    for (int s = 0; s < steps; s++) {
        const int ra = ra0 + s, rb = ra - h;
        const bool din = ra >= 0 && ra < H, dout = s >= h && rb >= 0;
        __syncwarp();  // every lane is done reading the previous staged rows
        if (din)
            commit(S.rin, pin, ra);
        if (dout)
            commit(S.rout, pout, rb);
        const int I = pc;
        if (s + 1 < steps)
            fetch(s + 1);
        __syncwarp();
        if (din) {
            uint32_t nb = 0;
#pragma unroll
            for (int e = 0; e < 7; e++) {
                const int a = S.rin[ok[e]];
                atomicAdd(&ownl[a * kOW], dplus);
                nb += (uint32_t)(a - Q) >> 31;  // a < Q
            }
            bown += nb;
#pragma unroll
            for (int t = 0; t < 3; t++) {
                if (gmask >> t & 1u) {
                    const int a = S.rin[gk[t]];
                    atomicAdd(&S.grp[G][a], 1u);
                    atomicAdd(&S.grpQ[G][a >> 2], 1u);
                }
            }
            for (int t = 0; CORE && t < core_rounds; t++) {
                const int e = lane + 32 * t;
                if (e < ncore) {
                    const int a = S.rin[31 + e];
                    atomicAdd(&S.core[a], 1u);
                    atomicAdd(&S.coreQ[G][a >> 2], 1u);
                }
            }
        }
        if (dout) {
            uint32_t nb = 0;
#pragma unroll
            for (int e = 0; e < 7; e++) {
                const int b = S.rout[ok[e]];
                atomicAdd(&ownl[b * kOW], dminus);
                nb += (uint32_t)(b - Q) >> 31;  // b < Q
            }
            bown -= nb;
#pragma unroll
            for (int t = 0; t < 3; t++) {
                if (gmask >> t & 1u) {
                    const int b = S.rout[gk[t]];
                    atomicAdd(&S.grp[G][b], 0xFFFFFFFFu);
                    atomicAdd(&S.grpQ[G][b >> 2], 0xFFFFFFFFu);
                }
            }
            for (int t = 0; CORE && t < core_rounds; t++) {
                const int e = lane + 32 * t;
                if (e < ncore) {
                    const int b = S.rout[31 + e];
                    atomicAdd(&S.core[b], 0xFFFFFFFFu);
                    atomicAdd(&S.coreQ[G][b >> 2], 0xFFFFFFFFu);
                }
            }
        }
        if (s < h - 1)
            continue;  // warm-up step (uniform)

        const int64_t i = y0 + s - h + 1;
        __syncwarp();
        // exclusive prefixes of the shared parts' 4-value totals
        if (has_grp) {
            // lane (G, pos) owns totals 8 pos .. 8 pos + 7 of group G
            const uint4 a = *reinterpret_cast<const uint4 *>(&S.grpQ[G][8 * pos]);
            const uint4 b = *reinterpret_cast<const uint4 *>(&S.grpQ[G][8 * pos + 4]);
            const uint32_t p0 = a.x, p1 = p0 + a.y, p2 = p1 + a.z, p3 = p2 + a.w;
            const uint32_t p4 = p3 + b.x, p5 = p4 + b.y, p6 = p5 + b.z, p7 = p6 + b.w;
            uint32_t sc = p7;
#pragma unroll
            for (int d = 1; d < 8; d <<= 1) {
                const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, sc, d, 8);
                if (pos >= d)
                    sc += v;
            }
            const uint32_t ex = sc - p7;
            *reinterpret_cast<uint4 *>(&S.cumGrp[G][8 * pos]) = make_uint4(ex, ex + p0, ex + p1, ex + p2);
            *reinterpret_cast<uint4 *>(&S.cumGrp[G][8 * pos + 4]) =
                make_uint4(ex + p3, ex + p4, ex + p5, ex + p6);
            if (pos == 7)
                S.cumGrp[G][64] = sc;
        }
        if (CORE) {
            // lane L owns totals 2 L, 2 L + 1 (summed over the four partials)
            uint32_t v0 = 0, v1 = 0;
#pragma unroll
            for (int gg = 0; gg < 4; gg++) {
                const uint2 a = *reinterpret_cast<const uint2 *>(&S.coreQ[gg][2 * lane]);
                v0 += a.x;
                v1 += a.y;
            }
            uint32_t sc = v0 + v1;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, sc, d);
                if (lane >= d)
                    sc += v;
            }
            const uint32_t ex = sc - v0 - v1;
            *reinterpret_cast<uint2 *>(&S.cumCore[2 * lane]) = make_uint2(ex, ex + v0);
            if (lane == 31)
                S.cumCore[64] = sc;
        }
        __syncwarp();
        // lanes past the image's last column take part in the warp-wide
        // loop below with nothing to move
        uint32_t below = 0;
        bool more_up = false, more_down = false;
        uint32_t o[4], c[4];
        auto counts = [&](int v0) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int v = v0 + k;
                v = v < 0 ? 0 : v;
                o[k] = own_count(ownl[v * kOW]);
                c[k] = o[k];
                if (has_grp)
                    c[k] += S.grp[G][v];
                if (CORE)
                    c[k] += S.core[v];
            }
        };
        if (live) {
            const int rows = (int)((i + win.u < g.H - 1 ? i + win.u : g.H - 1) -
                                   (i - win.o > -1 ? i - win.o : -1));
            if (rows != rows_prev) {
                rows_prev = rows;
                const int64_t n = (int64_t)rows * (cols > 0 ? cols : 1);
                int64_t r = (n * (int64_t)q_num + q_den - 1) / q_den;
                if (r < 1)
                    r = 1;
                if (r > n)
                    r = n;
                rho = (uint32_t)r;
            }
            below = bown;
            if (has_grp)
                below += q_part_below(S.grp[G], S.cumGrp[G], Q);
            if (CORE)
                below += q_part_below(S.core, S.cumCore, Q);
            // counts at Q - 2 .. Q + 1 settle moves of up to two gray values
            // (predicated, no branches); longer moves repeat four-value
            // rounds while any lane of the warp still needs one
            counts(Q - 2);
            const uint32_t bp1 = below + c[2], bm1 = below - c[1];
            const bool up1 = Q < 255 && bp1 < rho;
            const bool up2 = up1 && Q + 1 < 255 && bp1 + c[3] < rho;
            const bool dn1 = Q > 0 && below >= rho;
            const bool dn2 = dn1 && Q - 1 > 0 && bm1 >= rho;
            bown += (up1 ? o[2] : 0u) + (up2 ? o[3] : 0u) - (dn1 ? o[1] : 0u) - (dn2 ? o[0] : 0u);
            below = up2 ? bp1 + c[3] : up1 ? bp1 : dn2 ? bm1 - c[0] : dn1 ? bm1 : below;
            Q += (up1 ? 1 : 0) + (up2 ? 1 : 0) - (dn1 ? 1 : 0) - (dn2 ? 1 : 0);
            more_up = up2;
            more_down = dn2 && below >= rho;
        }
        while (__any_sync(0xFFFFFFFFu, more_up || more_down)) {
            // up: levels Q .. Q + 3; down: levels Q - 4 .. Q - 1
            counts(more_down ? Q - 4 : Q);
            int k = 0;
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const uint32_t cu = c[t], ou = o[t], cd = c[3 - t], od = o[3 - t];
                const bool su = more_up && k == t && Q + t < 255 && below + cu < rho;
                const bool sd = more_down && k == t && Q - t > 0 && below >= rho;
                below = su ? below + cu : sd ? below - cd : below;
                bown = su ? bown + ou : sd ? bown - od : bown;
                k = (su || sd) ? t + 1 : k;
            }
            Q += more_up ? k : -k;
            more_up = more_up && k == 4;
            more_down = more_down && k == 4 && below >= rho;
        }
        uint32_t bit = 0;
        if (live) {
            bit = (I <= Q - offset) ? 0u : 1u;
            if (Qout && BZ_DBG_IN(Qout + i * g.W + j, 1, Qout, (size_t)(g.H * g.W), kDbgOutput))
                Qout[i * g.W + j] = (uint8_t)Q;
        }
        if (out) {
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
            if (lane < 4) {
                const int64_t c8 = x0 + 8 * lane;
                if (c8 < g.W && BZ_DBG_IN(out + i * out_pitch + (c8 >> 3), 1, out,
                                          dbg_extent(g.H, out_pitch, (g.W + 7) / 8), kDbgOutput))
                    out[i * out_pitch + (c8 >> 3)] = (uint8_t)(word >> (8 * lane));
            }
        }
    }
}

}  // namespace bz
