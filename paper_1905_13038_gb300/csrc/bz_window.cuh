// Window-statistics + local-threshold tile routine (device side).
//
// One warp computes one tile of 256 output columns x `rows` output rows.
// Lane t owns the 8 output columns j = x0 + 8t .. x0 + 8t + 7.
//
// Formulation (Sec. 3.1 identities applied at both window edges):
//   C_b(i)  = sum of I over rows (i-o, i+u] in column b   (stripe level)
//   E_j(i)  = C_{j+r}(i) - C_{j-l}(i)                      (window level step)
//   S1(i,j) = S1(i, j-1) + E_j(i)                            (first identity)
//   E_j(i)  = E_j(i-1) + I[i+u][j+r] - I[i+u][j-l]
//                       - I[i-o][j+r] + I[i-o][j-l]          (second identity)
// and the same with I^2 for S2.  Each lane keeps E for its 8 columns in
// registers and slides them down the tile (4 byte streams per row); the
// window sums of a row are then a prefix sum of E along the row: a lane-local
// prefix plus a warp scan, offset by the anchor S(i, x0-1), which the warp
// itself slides down with DP4A row sums over the anchor window.  There is no
// shared memory, no halo column and no block-level synchronisation.
//
// Threshold: certified FP32 evaluation of the canonical formula with a
// rigorous absolute error bound E; pixels with |I - t32| <= E are evaluated
// with the canonical FP64 sequence, so BZ_FP64 output equals the canonical
// FP64 decision bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bz {

constexpr int kColsPerLane = 8;
constexpr int kTileCols = 32 * kColsPerLane;  // 256

enum Mode : int { MODE_FP64 = 0, MODE_FP32 = 1, MODE_FP64_DIRECT = 2, MODE_SUMS = 3, MODE_REPORT = 4 };

struct Image {
    const uint8_t *img;
    int64_t H, W, pitch;
};

struct Window {
    int h, w, l, r, o, u;
};

// t = alpha*m + (beta*m + gamma)*s ; Sauvola: alpha = 1-k, beta = k/R,
// gamma = 0 ; Niblack: alpha = 1, beta = 0, gamma = k.
struct Thresh {
    float alpha, beta, gamma;
    float aalpha, abeta, agamma;
    float eps;      // relative part of the certified bound
    float delta64;  // absolute bound on |t64 - t_exact|
    double k, R;    // canonical FP64 parameters
    int method;     // 0 Sauvola, 1 Niblack
};

struct Outputs {
    uint8_t *bits;        // packed output (binarize modes)
    int64_t out_pitch;
    uint32_t *S1;         // MODE_SUMS (each may be null)
    uint64_t *S2;
    uint32_t *n;
    unsigned long long *fallbacks;  // optional FP64-fallback counter
    unsigned long long *flips;      // MODE_REPORT
    unsigned long long *maxdt_bits; // MODE_REPORT (double bits, >= 0)
};

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= d)
            v += y;
    }
    return v;
}

// ------------------------------------------------------------ threshold --
// Canonical FP64 threshold: IEEE binary64, round to nearest, no contraction,
// in the documented order.
__device__ __forceinline__ double canonical_t(int method, uint32_t S1, uint64_t S2, uint32_t n,
                                              double k, double R)
{
    const long long V = (long long)n * (long long)S2 - (long long)S1 * (long long)S1;
    const double nd = __uint2double_rn(n);
    const double m = __ddiv_rn(__uint2double_rn(S1), nd);
    const double s = __dsqrt_rn(__ddiv_rn(__ll2double_rn(V), __dmul_rn(nd, nd)));
    if (method == 0)
        return __dmul_rn(m, __dadd_rn(1.0, __dmul_rn(k, __dadd_rn(__ddiv_rn(s, R), -1.0))));
    return __dadd_rn(m, __dmul_rn(k, s));
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------ the tile --
// Byte m (0..7) of an 8-byte group, zero-extended.
__device__ __forceinline__ int32_t byte_at(uint2 v, int m)
{
    return (int32_t)__byte_perm(m < 4 ? v.x : v.y, 0u, 0x4440u | (unsigned)(m & 3));
}

// 8 gray levels at columns col .. col+7 of the row starting at rp (which is
// an in-image row); columns outside [0, W) read as 0.  `fast`: the 8 bytes
// lie inside the row and VEC alignment holds; k = col & 7 (warp-uniform);
// sel = byte_perm selector for offset k & 3.
template <bool VEC>
__device__ __forceinline__ uint2 ld8(const uint8_t *rp, int64_t col, bool fast, int k, unsigned sel,
                                     int64_t W)
{
    if (VEC && fast) {
        const uint8_t *p = rp + (col - k);
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
        if (k == 0)
            return a;
        const uint2 b = __ldg(reinterpret_cast<const uint2 *>(p + 8));
        return k < 4 ? make_uint2(__byte_perm(a.x, a.y, sel), __byte_perm(a.y, b.x, sel))
                     : make_uint2(__byte_perm(a.y, b.x, sel), __byte_perm(b.x, b.y, sel));
    }
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int64_t c = col + m;
        const uint32_t b = (c >= 0 && c < W) ? (uint32_t)rp[c] : 0u;
        if (m < 4)
            lo |= b << (8 * m);
        else
            hi |= b << (8 * (m - 4));
    }
    return make_uint2(lo, hi);
}

// Anchor row sums: this lane's share of the columns [c0, c0 + cnt) of one
// row, as (sum, sum of squares); words of 4 columns, lane-strided.
template <bool VEC>
__device__ __forceinline__ void anchor_words(const uint8_t *rp, int64_t a4, int64_t c0, int64_t end,
                                             int64_t W, int lane, uint32_t &s1, uint32_t &s2)
{
    for (int64_t c4 = a4 + 4 * lane; c4 < end; c4 += 128) {
        uint32_t wd;
        if (VEC && c4 >= 0 && c4 + 4 <= W) {
            wd = __ldg(reinterpret_cast<const uint32_t *>(rp + c4));
        } else {
            wd = 0;
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const int64_t c = c4 + m;
                if (c >= 0 && c < W)
                    wd |= (uint32_t)rp[c] << (8 * m);
            }
        }
        uint32_t keep = 0xFFFFFFFFu;
        if (c4 < c0)
            keep &= 0xFFFFFFFFu << (8 * (int)(c0 - c4));
        if (c4 + 4 > end)
            keep &= 0xFFFFFFFFu >> (8 * (int)(c4 + 4 - end));
        wd &= keep;
        s1 = __dp4a(wd, 0x01010101u, s1);
        s2 = __dp4a(wd, wd, s2);
    }
}

// Canonical FP64 decision for one pixel (kept out of line so that no FP64
// work is scheduled on the FP32 hot path).
static __device__ __noinline__ uint32_t fp64_bit(int method, uint32_t I, uint32_t S1, uint64_t S2,
                                          uint32_t n, double k, double R)
{
    return ((double)I <= canonical_t(method, S1, S2, n, k, R)) ? 0u : 1u;
}

// S2T: uint32_t when h*w <= 66051 (S2 < 2^32), else unsigned long long.
template <int MODE, bool VEC, typename S2T>
__device__ __forceinline__ void window_tile(const Image &g, const Window &win, const Thresh &T,
                                            const Outputs &o, int64_t x0, int64_t y0, int64_t y1,
                                            int lane)
{
    const int64_t W = g.W, H = g.H;
    const int64_t j0 = x0 + (int64_t)kColsPerLane * lane;
    const int l = win.l, r = win.r, oo = win.o, u = win.u;

    // ---- per-lane constants
    const int64_t colA = j0 + r, colB = j0 - l;  // entering / leaving edge columns
    const bool fastA = VEC && colA >= 0 && colA + 8 <= W;
    const bool fastB = VEC && colB >= 0 && colB + 8 <= W;
    const int kA = (int)(colA & 7), kB = (int)(colB & 7);  // warp-uniform
    const unsigned selA = (unsigned)(kA & 3) * 0x1111u + 0x3210u;
    const unsigned selB = (unsigned)(kB & 3) * 0x1111u + 0x3210u;
    const bool fastP = VEC && j0 + 8 <= W;

    uint32_t cols[kColsPerLane];
    float inv_cols[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        const int64_t j = j0 + m;
        const int64_t hi = j + r < W - 1 ? j + r : W - 1;
        const int64_t lo = j - l > -1 ? j - l : -1;
        const int64_t c = hi - lo;
        cols[m] = (uint32_t)(c < 1 ? 1 : c);  // c < 1 only for j >= W
        inv_cols[m] = __frcp_rn((float)cols[m]);
    }
    // anchor window: columns [x0-l, x0-1+r] (the window of column x0-1)
    const int64_t ac0 = x0 - l, aend = x0 + r;
    const int64_t a4 = ac0 >= 0 ? (ac0 & ~(int64_t)3) : -((-ac0 + 3) & ~(int64_t)3);

    // ---- warm-up: E and the anchor for row y0 (window rows (y0-o, y0+u])
    int32_t E1[kColsPerLane], E2[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        E1[m] = 0;
        E2[m] = 0;
    }
    uint32_t a1p = 0, a2p = 0;
    {
        int64_t a_lo = y0 - oo + 1, a_hi = y0 + u;
        if (a_lo < 0)
            a_lo = 0;
        if (a_hi > H - 1)
            a_hi = H - 1;
        for (int64_t a = a_lo; a <= a_hi; a++) {
            const uint8_t *rp = g.img + a * g.pitch;
            const uint2 A = ld8<VEC>(rp, colA, fastA, kA, selA, W);
            const uint2 B = ld8<VEC>(rp, colB, fastB, kB, selB, W);
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const int32_t av = byte_at(A, m), bv = byte_at(B, m);
                E1[m] += av - bv;
                E2[m] += av * av - bv * bv;
            }
            anchor_words<VEC>(rp, a4, ac0, aend, W, lane, a1p, a2p);
        }
    }
    uint32_t A1 = __reduce_add_sync(0xFFFFFFFFu, a1p);
    S2T A2;
    {
        unsigned long long v = (unsigned long long)a2p;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
        A2 = (S2T)v;
    }

    unsigned long long nfb = 0, nflip = 0;
    double maxdt = 0.0;

    // prefetched slide data for the next row
    uint2 nA = make_uint2(0, 0), nB = nA, nC = nA, nD = nA;
    uint32_t nd1 = 0, nd2 = 0;  // anchor increment partials (entering - leaving)
    auto prefetch = [&](int64_t i) {
        const int64_t ra = i + u, rb = i - oo;
        nA = nB = nC = nD = make_uint2(0, 0);
        uint32_t e1 = 0, e2 = 0, x1 = 0, x2 = 0;
        if (ra < H) {
            const uint8_t *rp = g.img + ra * g.pitch;
            nA = ld8<VEC>(rp, colA, fastA, kA, selA, W);
            nB = ld8<VEC>(rp, colB, fastB, kB, selB, W);
            anchor_words<VEC>(rp, a4, ac0, aend, W, lane, e1, e2);
        }
        if (rb >= 0) {
            const uint8_t *rp = g.img + rb * g.pitch;
            nC = ld8<VEC>(rp, colA, fastA, kA, selA, W);
            nD = ld8<VEC>(rp, colB, fastB, kB, selB, W);
            anchor_words<VEC>(rp, a4, ac0, aend, W, lane, x1, x2);
        }
        nd1 = e1 - x1;
        nd2 = e2 - x2;
    };
    if (y0 + 1 < y1)
        prefetch(y0 + 1);

    for (int64_t i = y0; i < y1; i++) {
        if (i > y0) {
            // slide every E and the anchor from row i-1 to row i
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const int32_t av = byte_at(nA, m), bv = byte_at(nB, m);
                const int32_t cv = byte_at(nC, m), dv = byte_at(nD, m);
                E1[m] += (av + dv) - (bv + cv);
                E2[m] += (av * av + dv * dv) - (bv * bv + cv * cv);
            }
            A1 += (uint32_t)__reduce_add_sync(0xFFFFFFFFu, nd1);
            A2 += (S2T)(int64_t)(int32_t)__reduce_add_sync(0xFFFFFFFFu, nd2);
            if (i + 1 < y1)
                prefetch(i + 1);
        }

        // window sums along the row: lane prefix + warp scan + anchor
        uint32_t p1[kColsPerLane];
        S2T p2[kColsPerLane];
        uint32_t run1 = 0;
        S2T run2 = (S2T)0u;
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            run1 += (uint32_t)E1[m];
            run2 += (S2T)(int64_t)E2[m];
            p1[m] = run1;
            p2[m] = run2;
        }
        const uint32_t inc1 = warp_incl_scan<uint32_t>(run1, lane);
        const S2T inc2 = warp_incl_scan<S2T>(run2, lane);
        const uint32_t off1 = A1 + (inc1 - run1);
        const S2T off2 = A2 + (inc2 - run2);

        const int64_t rows = (i + u < H - 1 ? i + u : H - 1) - (i - oo > -1 ? i - oo : -1);
        const uint32_t nrow = (uint32_t)rows;

        if (MODE == MODE_SUMS) {
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const int64_t j = j0 + m;
                if (j < W) {
                    const int64_t idx = i * W + j;
                    if (o.S1)
                        o.S1[idx] = off1 + p1[m];
                    if (o.S2)
                        o.S2[idx] = (uint64_t)(off2 + p2[m]);
                    if (o.n)
                        o.n[idx] = nrow * cols[m];
                }
            }
            continue;
        }

        const float inv_rows = __frcp_rn((float)rows);
        const uint8_t *prow = g.img + i * g.pitch;
        const uint2 P = ld8<VEC>(prow, j0, fastP, 0, 0x3210u, W);
        uint32_t byte = 0, undecided = 0;
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            const uint32_t S1 = off1 + p1[m];
            const uint64_t S2 = (uint64_t)(off2 + p2[m]);
            const uint32_t n = nrow * cols[m];
            uint32_t bit;
            if (MODE == MODE_FP64_DIRECT) {
                bit = fp64_bit(T.method, (uint32_t)byte_at(P, m), S1, S2, n, T.k, T.R);
            } else {
                // exact V = n S2 - S1^2 (< 2^48), converted from two 32-bit halves
                const uint64_t V = (uint64_t)n * S2 - (uint64_t)S1 * (uint64_t)S1;
                const float Vhi = __int_as_float(0x4B000000u | (uint32_t)(V >> 32)) - 8388608.0f;
                const float Vf = fmaf(Vhi, 4294967296.0f, __uint2float_rn((uint32_t)V));
                const float inv_n = inv_rows * inv_cols[m];
                const float mu = __uint2float_rn(S1) * inv_n;
                const float var = (Vf * inv_n) * inv_n;
                const float s = sqrt_approx(var);
                const float t = fmaf(fmaf(T.beta, mu, T.gamma), s, T.alpha * mu);
                // the pixel as a float: 2^23 + I from its byte, minus 2^23
                const float If =
                    __int_as_float(__byte_perm(m < 4 ? P.x : P.y, 0x4B000000u, 0x7440u | (unsigned)(m & 3))) -
                    8388608.0f;
                const float d = If - t;
                bit = d > 0.0f ? 1u : 0u;
                if (MODE == MODE_FP64) {
                    const float mag = fmaf(fmaf(T.abeta, mu, T.agamma), s, T.aalpha * mu);
                    const float E = fmaf(T.eps, mag, T.delta64);
                    undecided |= (fabsf(d) <= E ? 1u : 0u) << m;
                } else if (MODE == MODE_REPORT) {
                    if (j0 + m < W) {
                        const double t64 = canonical_t(T.method, S1, S2, n, T.k, T.R);
                        const uint32_t I = (uint32_t)byte_at(P, m);
                        const uint32_t b64 = ((double)I <= t64) ? 0u : 1u;
                        nflip += (b64 != bit);
                        const double dt = fabs((double)t - t64);
                        maxdt = dt > maxdt ? dt : maxdt;
                    }
                }
            }
            byte |= bit << m;
        }
        if (MODE == MODE_FP64) {
            // near-ties: canonical FP64 evaluation, off the hot path
            if (j0 + 8 > W)
                undecided &= (1u << (j0 < W ? W - j0 : 0)) - 1u;
            if (__any_sync(0xFFFFFFFFu, undecided != 0) && undecided) {
#pragma unroll
                for (int m = 0; m < kColsPerLane; m++) {
                    if (undecided >> m & 1u) {
                        const uint32_t b = fp64_bit(T.method, (uint32_t)byte_at(P, m), off1 + p1[m],
                                                    (uint64_t)(off2 + p2[m]), nrow * cols[m], T.k, T.R);
                        byte = (byte & ~(1u << m)) | (b << m);
                    }
                }
                nfb += __popc(undecided);
            }
        }
        if (MODE != MODE_REPORT && j0 < W) {
            if (j0 + 8 > W)
                byte &= (1u << (W - j0)) - 1u;  // padding bits are 0
            o.bits[i * o.out_pitch + (j0 >> 3)] = (uint8_t)byte;
        }
    }

    if (MODE == MODE_FP64 && o.fallbacks) {
        const unsigned v = __reduce_add_sync(0xFFFFFFFFu, (unsigned)nfb);
        if (lane == 0 && v)
            atomicAdd(o.fallbacks, (unsigned long long)v);
    }
    if (MODE == MODE_REPORT) {
        unsigned long long v = nflip;
        double mx = maxdt;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
            const double y = __shfl_xor_sync(0xFFFFFFFFu, mx, d);
            mx = y > mx ? y : mx;
        }
        if (lane == 0) {
            if (v)
                atomicAdd(o.flips, v);
            atomicMax(o.maxdt_bits, (unsigned long long)__double_as_longlong(mx));
        }
    }
}

}  // namespace bz
