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

// ---------------------------------------------------------------- loads --
// 8 gray levels of row `row`, columns col0 .. col0+7; 0 outside the image.
// VEC: image base and pitch are multiples of 8, so aligned 8-byte loads of
// the row never leave [row start, row start + pitch).
template <bool VEC>
__device__ __forceinline__ uint2 load8(const Image &g, int64_t row, int64_t col0)
{
    if (row < 0 || row >= g.H)
        return make_uint2(0u, 0u);
    const uint8_t *rp = g.img + row * g.pitch;
    if (VEC && col0 >= 0 && col0 + 8 <= g.W) {
        const int64_t a8 = col0 & ~(int64_t)7;
        const int k = (int)(col0 - a8);
        const uint2 p = __ldg(reinterpret_cast<const uint2 *>(rp + a8));
        if (k == 0)
            return p;
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(rp + a8 + 8));
        const unsigned sel = (unsigned)(k & 3) * 0x1111u + 0x3210u;
        uint2 v;
        if (k < 4) {
            v.x = __byte_perm(p.x, p.y, sel);
            v.y = __byte_perm(p.y, q.x, sel);
        } else {
            v.x = __byte_perm(p.y, q.x, sel);
            v.y = __byte_perm(q.x, q.y, sel);
        }
        return v;
    }
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int64_t c = col0 + m;
        const uint32_t b = (c >= 0 && c < g.W) ? (uint32_t)rp[c] : 0u;
        if (m < 4)
            lo |= b << (8 * m);
        else
            hi |= b << (8 * (m - 4));
    }
    return make_uint2(lo, hi);
}

// 4 gray levels at columns c4 .. c4+3 (c4 a multiple of 4), 0 outside.
template <bool VEC>
__device__ __forceinline__ uint32_t load4_aligned(const Image &g, int64_t row, int64_t c4)
{
    if (row < 0 || row >= g.H)
        return 0u;
    const uint8_t *rp = g.img + row * g.pitch;
    if (VEC && c4 >= 0 && c4 + 4 <= g.W)
        return __ldg(reinterpret_cast<const uint32_t *>(rp + c4));
    uint32_t v = 0;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int64_t c = c4 + m;
        if (c >= 0 && c < g.W)
            v |= (uint32_t)rp[c] << (8 * m);
    }
    return v;
}

__device__ __forceinline__ uint32_t byte_of(uint2 v, int m)
{
    return ((m < 4 ? v.x : v.y) >> (8 * (m & 3))) & 0xFFu;
}

// Sum and sum of squares of row `row` over columns [c0, c0 + cnt), spread
// over the warp (each lane returns its partial; caller reduces).
template <bool VEC>
__device__ __forceinline__ void row_partial(const Image &g, int64_t row, int64_t c0, int cnt,
                                            int lane, uint32_t &s1, uint32_t &s2)
{
    if (row < 0 || row >= g.H || cnt <= 0)
        return;
    const int64_t a4 = c0 >= 0 ? (c0 & ~(int64_t)3) : -((-c0 + 3) & ~(int64_t)3);
    const int64_t end = c0 + cnt;  // exclusive
    for (int64_t c4 = a4 + 4 * lane; c4 < end; c4 += 128) {
        uint32_t wd = load4_aligned<VEC>(g, row, c4);
        // keep only the bytes whose column lies in [c0, end)
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

__device__ __forceinline__ int32_t warp_allsum(int32_t v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
    return v;
}

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

struct Decision {
    uint32_t bit;       // 0/1 decision
    bool certain;       // decision certified equal to the canonical FP64 one
    float t32;          // FP32 threshold (report mode)
};

// FP32 evaluation of the threshold from the exact integers, with the
// certified margin.
__device__ __forceinline__ Decision decide_f32(const Thresh &T, uint32_t I, uint32_t S1, long long V,
                                               float inv_n)
{
    const float S1f = __uint2float_rn(S1);
    const float Vf = __ll2float_rn(V);
    const float m = S1f * inv_n;
    const float var = (Vf * inv_n) * inv_n;
    const float s = sqrt_approx(var);
    const float g = fmaf(T.beta, m, T.gamma);
    const float t = fmaf(g, s, T.alpha * m);
    const float mag = fmaf(fmaf(T.abeta, m, T.agamma), s, T.aalpha * m);
    const float E = fmaf(T.eps, mag, T.delta64);
    const float If = __uint2float_rn(I);
    Decision d;
    d.t32 = t;
    d.bit = If > t ? 1u : 0u;
    d.certain = (If > t + E) || (If < t - E);
    return d;
}

// ------------------------------------------------------------ the tile --
// S2T: uint32_t when h*w <= 66051 (S2 < 2^32), else unsigned long long.
template <int MODE, bool VEC, typename S2T>
__device__ __forceinline__ void window_tile(const Image &g, const Window &win, const Thresh &T,
                                            const Outputs &o, int64_t x0, int64_t y0, int64_t y1,
                                            int lane)
{
    const int64_t j0 = x0 + (int64_t)kColsPerLane * lane;
    const int l = win.l, r = win.r, oo = win.o, u = win.u;

    // per-column clipped widths and their reciprocals (Algorithm 1 count)
    uint32_t cols[kColsPerLane];
    float inv_cols[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        const int64_t j = j0 + m;
        int64_t hi = j + r < g.W - 1 ? j + r : g.W - 1;
        int64_t lo = j - l > -1 ? j - l : -1;
        int64_t c = hi - lo;
        if (c < 1)
            c = 1;  // only for j >= W (outputs discarded)
        cols[m] = (uint32_t)c;
        inv_cols[m] = __frcp_rn((float)c);
    }

    // warm-up: E over the window rows of y0, and the anchor S(y0, x0-1)
    int32_t E1[kColsPerLane], E2[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        E1[m] = 0;
        E2[m] = 0;
    }
    uint32_t a1p = 0, a2p = 0;  // lane partials of the anchor
    const int64_t ac0 = x0 - l;  // anchor window columns [x0-l, x0-1+r]
    const int aw = win.w;
    for (int64_t a = y0 - oo + 1; a <= y0 + u; a++) {
        if (a < 0 || a >= g.H)
            continue;
        const uint2 A = load8<VEC>(g, a, j0 + r);
        const uint2 B = load8<VEC>(g, a, j0 - l);
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            const int32_t av = (int32_t)byte_of(A, m), bv = (int32_t)byte_of(B, m);
            E1[m] += av - bv;
            E2[m] += av * av - bv * bv;
        }
        row_partial<VEC>(g, a, ac0, aw, lane, a1p, a2p);
    }
    S2T A2 = (S2T)(uint32_t)0;
    uint32_t A1 = (uint32_t)warp_allsum((int32_t)a1p);
    {
        // a2 partials may exceed int32 when summed over h rows: reduce in 64 bits
        unsigned long long v = (unsigned long long)(uint32_t)a2p;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
        A2 = (S2T)v;
    }

    unsigned long long nfb = 0, nflip = 0;
    double maxdt = 0.0;

    for (int64_t i = y0; i < y1; i++) {
        if (i > y0) {
            // slide every E and the anchor from row i-1 to row i
            const int64_t ra = i + u, rb = i - oo;
            const uint2 A = load8<VEC>(g, ra, j0 + r);
            const uint2 B = load8<VEC>(g, ra, j0 - l);
            const uint2 C = load8<VEC>(g, rb, j0 + r);
            const uint2 D = load8<VEC>(g, rb, j0 - l);
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const int32_t av = (int32_t)byte_of(A, m), bv = (int32_t)byte_of(B, m);
                const int32_t cv = (int32_t)byte_of(C, m), dv = (int32_t)byte_of(D, m);
                E1[m] += (av - bv) - (cv - dv);
                E2[m] += (av * av - bv * bv) - (cv * cv - dv * dv);
            }
            uint32_t d1 = 0, d2 = 0, e1 = 0, e2 = 0;
            row_partial<VEC>(g, ra, ac0, aw, lane, d1, d2);
            row_partial<VEC>(g, rb, ac0, aw, lane, e1, e2);
            A1 += (uint32_t)warp_allsum((int32_t)(d1 - e1));
            A2 += (S2T)(int64_t)warp_allsum((int32_t)(d2 - e2));
        }

        // window sums along the row: lane prefix + warp scan + anchor
        uint32_t p1[kColsPerLane];
        S2T p2[kColsPerLane];
        uint32_t run1 = 0;
        S2T run2 = (S2T)(uint32_t)0;
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

        const int64_t rows = (i + u < g.H - 1 ? i + u : g.H - 1) - (i - oo > -1 ? i - oo : -1);
        const float inv_rows = __frcp_rn((float)rows);

        if (MODE == MODE_SUMS) {
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const int64_t j = j0 + m;
                if (j < g.W) {
                    const int64_t idx = i * g.W + j;
                    if (o.S1)
                        o.S1[idx] = off1 + p1[m];
                    if (o.S2)
                        o.S2[idx] = (uint64_t)(off2 + p2[m]);
                    if (o.n)
                        o.n[idx] = (uint32_t)rows * cols[m];
                }
            }
            continue;
        }

        const uint2 P = load8<VEC>(g, i, j0);  // the pixels themselves
        uint32_t byte = 0;
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            const int64_t j = j0 + m;
            const uint32_t S1 = off1 + p1[m];
            const uint64_t S2 = (uint64_t)(off2 + p2[m]);
            const uint32_t n = (uint32_t)rows * cols[m];
            const uint32_t I = byte_of(P, m);
            const long long V = (long long)n * (long long)S2 - (long long)S1 * (long long)S1;
            uint32_t bit;
            if (MODE == MODE_FP64_DIRECT) {
                bit = ((double)I <= canonical_t(T.method, S1, S2, n, T.k, T.R)) ? 0u : 1u;
            } else {
                const Decision d = decide_f32(T, I, S1, V, inv_rows * inv_cols[m]);
                bit = d.bit;
                if (MODE == MODE_FP64) {
                    if (!d.certain && j < g.W) {
                        bit = ((double)I <= canonical_t(T.method, S1, S2, n, T.k, T.R)) ? 0u : 1u;
                        nfb++;
                    }
                } else if (MODE == MODE_REPORT) {
                    if (j < g.W) {
                        const double t64 = canonical_t(T.method, S1, S2, n, T.k, T.R);
                        const uint32_t b64 = ((double)I <= t64) ? 0u : 1u;
                        nflip += (b64 != d.bit);
                        const double dt = fabs((double)d.t32 - t64);
                        maxdt = dt > maxdt ? dt : maxdt;
                    }
                }
            }
            if (j < g.W)
                byte |= bit << m;
        }
        if (MODE != MODE_REPORT && j0 < g.W)
            o.bits[i * o.out_pitch + (j0 >> 3)] = (uint8_t)byte;
    }

    if (MODE == MODE_FP64 && o.fallbacks) {
        unsigned long long v = nfb;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
        if (lane == 0 && v)
            atomicAdd(o.fallbacks, v);
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
