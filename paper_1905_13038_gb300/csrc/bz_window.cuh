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
// block-level synchronisation: the generic row routine uses no shared memory,
// the pipelined one (window_rows_pipe) only the warp's own (row slots of
// window sums, the column sums of its warm-up, tables, parked state).
//
// Threshold: certified FP32 evaluation of the canonical formula with a
// rigorous absolute error bound E; pixels with |I - t32| <= E are evaluated
// with the canonical FP64 sequence, so BZ_FP64 output equals the canonical
// FP64 decision bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bz_debug.cuh"

namespace bz {

constexpr int kColsPerLane = 8;
constexpr int kTileCols = 32 * kColsPerLane;  // 256
constexpr int kWarmRows = 8;                   // warm-up rows per batch (WARMB), a multiple of 4
// Per-warp shared memory of the pipelined path, in 16-byte units: two 2 KB
// row slots of window sums, the 2 KB edge column table, the 512-byte FP64
// near-tie list, the 1 KB table of per-row threshold constants, then 3.75 KB
// where the row loop parks its state while a near-tie row is decided.
constexpr int kPipeSlotsRows = 416;
constexpr int kPipeSlotsPark = kPipeSlotsRows + 64;
constexpr int kPipeParkWords = 30;                                 // per lane
constexpr int kPipeSlots = kPipeSlotsPark + kPipeParkWords * 8;  // 11.25 KB

enum Mode : int { MODE_FP64 = 0, MODE_FP32 = 1, MODE_FP64_DIRECT = 2, MODE_SUMS = 3, MODE_REPORT = 4 };

struct Image {
    const uint8_t *img;
    int64_t H, W, pitch;
};

// Bytes of an image buffer: H rows of pitch bytes (the C ABI's contract;
// aligned 8-byte loads may read a row's padding past column W).
__host__ __device__ inline size_t dbg_image_extent(const Image &g)
{
    return (size_t)(g.H * g.pitch);
}

struct Window {
    int h, w, l, r, o, u;
};

__device__ __forceinline__ float sqrt_approx(float x);
}  // namespace bz
#include "bz_table1.cuh"
namespace bz {

// t = alpha*m + (beta*m + gamma)*s ; Sauvola: alpha = 1-k, beta = k/R,
// gamma = 0 ; Niblack: alpha = 1, beta = 0, gamma = k.
struct Thresh {
    float alpha, beta, gamma;
    float aalpha, abeta, agamma;
    float eps;      // relative part of the certified bound
    float delta64;  // absolute bound on |t64 - t_exact|
    float bnd_c;    // interior pipelined form: bound on |d32 - (t64 - I)| over all pixels
    double k, R;    // canonical FP64 parameters
    int method;     // a bz::Method other than METHOD_QUANTILE
};

// The other Table 1 methods add their parameters and the global sums (kept
// out of Thresh so that the batched work list does not grow).
struct ThreshExt : Thresh {
    ExtParams X;           // Feng and Phansalkar parameters
    const GStats *gs;      // global sums (Wolf, Feng, Rais, Phansalkar)
    unsigned long long N;  // pixels of the image, for the global statistics
};

struct Outputs {
    uint8_t *bits;        // packed output (binarize modes)
    int64_t out_pitch;
    int64_t out_row0;     // image row i is output row i - out_row0
    int64_t out_byte0;    // image column j goes to output byte j / 8 - out_byte0
    size_t bits_bytes;    // extent of `bits` (bounds checks of the debug build)
    int64_t sums_n;       // elements of S1, S2 and n (debug build)
    uint32_t *S1;         // MODE_SUMS (each may be null)
    uint64_t *S2;
    uint32_t *n;
    unsigned long long *fallbacks;  // optional FP64-fallback counter
    unsigned long long *fallbacks_clear;  // the other call slot's counter, zeroed by the launch (after its wait)
    unsigned long long *flips;      // MODE_REPORT (each may be null)
    unsigned long long *maxdt_bits; // MODE_REPORT (double bits, >= 0)
    unsigned long long *maxratio_bits;  // MODE_REPORT: max |t32 - t64| / certified bound (double bits)
    int32_t report_path;  // MODE_REPORT: the path a BZ_FP32 launch takes (kReport*), whose form the flips follow
};

__device__ __forceinline__ void fallbacks_clear(const Outputs &o)
{
    if (o.fallbacks_clear && blockIdx.x == 0 && threadIdx.x == 0)
        *o.fallbacks_clear = 0ull;
}

// Paths of an FP32 binarize launch; MODE_REPORT counts flips with the FP32
// form of the path the same image and window take in BZ_FP32.
constexpr int32_t kReportGeneric = 0, kReportPipe = 1, kReportSmall = 2;

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

// Programmatic dependent launch: the kernels of a binarization call are
// launched so that each may be scheduled while the previous kernel in the
// stream drains (launch_pdl).  A kernel first lets its own dependents be
// scheduled, then waits until the previous grid has completed and its memory
// is visible; nothing is read before that wait.  Without the launch attribute
// both instructions are no-ops.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Single-image calls alternate between two FP64-fallback counters: a call
// counts into one and its launches zero the other for the next call, after
// their griddepcontrol.wait (the next call's kernels add only after their
// own wait, i.e. after this launch has finished), so that no memset sits
// between two launches and the next kernel can start early.
__device__ __forceinline__ void fallbacks_clear(const struct Outputs &o);

// ------------------------------------------------------------ threshold --
// Canonical FP64 threshold: IEEE binary64, round to nearest, no contraction,
// in the documented order.
__device__ __forceinline__ double canonical_t(int method, uint32_t S1, uint64_t S2, uint32_t n,
                                              double k, double R)
{
    const long long V = (long long)n * (long long)S2 - (long long)S1 * (long long)S1;
    if (V == 0) {
        // every in-image pixel of the window has the value S1 / n (equality
        // in the Cauchy-Schwarz inequality n S2 >= S1^2), so the canonical
        // sequence has m = S1 / n exactly, v = s = +0 and 0/R = +0: no
        // division or square root is left (the same doubles as below)
        const double m = __uint2double_rn(S1 / n);
        if (method == 0)
            return __dmul_rn(m, __dadd_rn(1.0, __dmul_rn(k, -1.0)));
        return __dadd_rn(m, __dmul_rn(k, 0.0));
    }
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
                                     int64_t W, const uint8_t *base = nullptr, size_t ext = 0)
{
    if (VEC && fast) {
        const uint8_t *p = rp + (col - k);
        if (!BZ_DBG_IN(p, k ? 16 : 8, base, ext, kDbgImage))
            return make_uint2(0u, 0u);
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
                                             int64_t W, int lane, uint32_t &s1, uint32_t &s2,
                                             const uint8_t *base = nullptr, size_t ext = 0)
{
    for (int64_t c4 = a4 + 4 * lane; c4 < end; c4 += 128) {
        uint32_t wd;
        if (VEC && c4 >= 0 && c4 + 4 <= W) {
            wd = BZ_DBG_IN(rp + c4, 4, base, ext, kDbgImage) ? __ldg(reinterpret_cast<const uint32_t *>(rp + c4))
                                                             : 0u;
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

// The same for the other Table 1 methods (scalars only, so that nothing is
// spilled to local memory for the call).
static __device__ __noinline__ uint32_t fp64_bit_ext(int method, uint32_t I, uint32_t S1, uint64_t S2,
                                                     uint32_t n, double k, double R, double alpha1,
                                                     double k1, double k2, double gamma, double p,
                                                     double q, double L, double M, double S)
{
    ExtParams X;
    X.alpha1 = alpha1;
    X.k1 = k1;
    X.k2 = k2;
    X.gamma = gamma;
    X.p = p;
    X.q = q;
    Global G;
    G.L = L;
    G.M = M;
    G.S = S;
    return ((double)I <= canonical_t_ext(method, S1, S2, n, k, R, X, G)) ? 0u : 1u;
}

// ---- packed-byte arithmetic for the E slide (two columns per step) ------
// dp2a.lo/hi with an unsigned 16-bit pair operand and unsigned bytes.
__device__ __forceinline__ uint32_t dp2a_lo_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp2a.lo.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t dp2a_hi_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp2a.hi.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// dp4a with unsigned bytes a and signed byte weights b.
__device__ __forceinline__ int32_t dp4a_us(uint32_t a, uint32_t b, int32_t c)
{
    int32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// E1 += a + d - b - c ; E2 += a^2 + d^2 - b^2 - c^2 for the 8 columns
// of a lane, from the byte groups A (row i+u, col j+r), B (row i+u, col j-l),
// C (row i-o, col j+r), D (row i-o, col j-l).
__device__ __forceinline__ void slide8(uint2 A, uint2 B, uint2 C, uint2 D, int32_t *E1,
                                       uint32_t *E2)
{
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const uint32_t Aw = q ? A.y : A.x, Bw = q ? B.y : B.x;
        const uint32_t Cw = q ? C.y : C.x, Dw = q ? D.y : D.x;
#pragma unroll
        for (int b = 0; b < 4; b += 2) {
            const int m = 4 * q + b;
            const unsigned sel = (unsigned)b | (unsigned)(4 + b) << 4 | (unsigned)(b + 1) << 8 |
                                 (unsigned)(5 + b) << 12;
            const uint32_t AD = __byte_perm(Aw, Dw, sel);  // a_m d_m a_m+1 d_m+1
            const uint32_t BC = __byte_perm(Bw, Cw, sel);  // b_m c_m b_m+1 c_m+1
            E2[m] = dp2a_lo_uu(__byte_perm(AD, 0u, 0x4140u), AD, E2[m]) -
                    dp2a_lo_uu(__byte_perm(BC, 0u, 0x4140u), BC, 0u);
            E2[m + 1] = dp2a_hi_uu(__byte_perm(AD, 0u, 0x4342u), AD, E2[m + 1]) -
                        dp2a_hi_uu(__byte_perm(BC, 0u, 0x4342u), BC, 0u);
            E1[m] = dp4a_us(BC, 0x0000FFFFu, dp4a_us(AD, 0x00000101u, E1[m]));
            E1[m + 1] = dp4a_us(BC, 0xFFFF0000u, dp4a_us(AD, 0x01010000u, E1[m + 1]));
        }
    }
}

// Four warm-up rows at once: the bytes of each column in rows r .. r+3 are
// gathered into one word (a 4 x 4 byte transpose, eight byte permutes per
// four columns and stream), so that E1 += sum (a - b) and E2 += sum (a^2 - b^2)
// take four DP4A per column instead of four extractions and updates per row.
__device__ __forceinline__ void warm8x4(const uint2 (&A)[4], const uint2 (&B)[4], int32_t *E1, uint32_t *E2)
{
#pragma unroll
    for (int q = 0; q < 2; q++) {
        uint32_t ca[4], cb[4];
        {
            const uint32_t a0 = q ? A[0].y : A[0].x, a1 = q ? A[1].y : A[1].x;
            const uint32_t a2 = q ? A[2].y : A[2].x, a3 = q ? A[3].y : A[3].x;
            const uint32_t lo01 = __byte_perm(a0, a1, 0x5140u), hi01 = __byte_perm(a0, a1, 0x7362u);
            const uint32_t lo23 = __byte_perm(a2, a3, 0x5140u), hi23 = __byte_perm(a2, a3, 0x7362u);
            ca[0] = __byte_perm(lo01, lo23, 0x5410u);
            ca[1] = __byte_perm(lo01, lo23, 0x7632u);
            ca[2] = __byte_perm(hi01, hi23, 0x5410u);
            ca[3] = __byte_perm(hi01, hi23, 0x7632u);
        }
        {
            const uint32_t b0 = q ? B[0].y : B[0].x, b1 = q ? B[1].y : B[1].x;
            const uint32_t b2 = q ? B[2].y : B[2].x, b3 = q ? B[3].y : B[3].x;
            const uint32_t lo01 = __byte_perm(b0, b1, 0x5140u), hi01 = __byte_perm(b0, b1, 0x7362u);
            const uint32_t lo23 = __byte_perm(b2, b3, 0x5140u), hi23 = __byte_perm(b2, b3, 0x7362u);
            cb[0] = __byte_perm(lo01, lo23, 0x5410u);
            cb[1] = __byte_perm(lo01, lo23, 0x7632u);
            cb[2] = __byte_perm(hi01, hi23, 0x5410u);
            cb[3] = __byte_perm(hi01, hi23, 0x7632u);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int m = 4 * q + c;
            E1[m] = dp4a_us(cb[c], 0xFFFFFFFFu, dp4a_us(ca[c], 0x01010101u, E1[m]));
            E2[m] = __dp4a(ca[c], ca[c], E2[m]) - __dp4a(cb[c], cb[c], 0u);
        }
    }
}

// Warm-up step: E1 += a - b ; E2 += a^2 - b^2 (entering rows only).
__device__ __forceinline__ void warm8(uint2 A, uint2 B, int32_t *E1, uint32_t *E2)
{
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const uint32_t Aw = q ? A.y : A.x, Bw = q ? B.y : B.x;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int m = 4 * q + b;
            const int32_t av = (int32_t)__byte_perm(Aw, 0u, 0x4440u | (unsigned)b);
            const int32_t bv = (int32_t)__byte_perm(Bw, 0u, 0x4440u | (unsigned)b);
            E1[m] += av - bv;
            E2[m] += (uint32_t)((av - bv) * (av + bv));
        }
    }
}

// 8 bytes at p (p - k4 is 4-byte aligned, k4 = byte offset in 0..3, sel the
// matching byte_perm selector), from three aligned 32-bit loads and no branch.
// The third word is only needed when k4 > 0; when k4 == 0 the second word is
// read again, so no byte past p + 8 is touched.  Requires image base and
// pitch to be multiples of 4 and the 8 bytes to lie inside the row.
__device__ __forceinline__ uint2 ld8_w3(const uint8_t *p, int k4, unsigned sel, const uint8_t *base = nullptr,
                                        size_t ext = 0)
{
    if (!BZ_DBG_IN(p - k4, k4 ? 12 : 8, base, ext, kDbgImage))
        return make_uint2(0u, 0u);
    const uint32_t *q = reinterpret_cast<const uint32_t *>(p - k4);
    const uint32_t w0 = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + (k4 ? 2 : 1));
    return make_uint2(__byte_perm(w0, w1, sel), __byte_perm(w1, w2, sel));
}

// Interior loads: 8 bytes at `p` (p - k is 8-byte aligned; k warp-uniform).
__device__ __forceinline__ uint2 ld8_fast(const uint8_t *p, int k, unsigned sel, const uint8_t *base = nullptr,
                                          size_t ext = 0)
{
    if (!BZ_DBG_IN(p - k, k ? 16 : 8, base, ext, kDbgImage))
        return make_uint2(0u, 0u);
    const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p - k));
    if (k == 0)
        return a;
    const uint2 b = __ldg(reinterpret_cast<const uint2 *>(p - k + 8));
    return k < 4 ? make_uint2(__byte_perm(a.x, a.y, sel), __byte_perm(a.y, b.x, sel))
                 : make_uint2(__byte_perm(a.y, b.x, sel), __byte_perm(b.x, b.y, sel));
}

// The pixel byte m of P as a float (2^23 + I, minus 2^23).
__device__ __forceinline__ float pixel_f(uint2 P, int m)
{
    return __int_as_float(__byte_perm(m < 4 ? P.x : P.y, 0x4B000000u, 0x7440u | (unsigned)(m & 3))) -
           8388608.0f;
}

// V = n S2 - S1^2 (exact, < 2^53) as a float, from 32-bit halves.  When
// S2 < 2^32 (h*w <= 66051) V < 2^47, so the high half is < 2^23 and converts
// exactly through the float bit pattern 2^23 + hi.
template <typename S2T>
__device__ __forceinline__ float v_float(uint32_t n, uint64_t S2, uint32_t S1)
{
    const uint64_t V = (uint64_t)n * S2 - (uint64_t)S1 * (uint64_t)S1;
    const uint32_t hi = (uint32_t)(V >> 32);
    const float fhi = sizeof(S2T) == 4 ? __int_as_float(0x4B000000u | hi) - 8388608.0f
                                       : __uint2float_rn(hi);
    return fmaf(fhi, 4294967296.0f, __uint2float_rn((uint32_t)V));
}

// The 8 pixels of one lane and row with a Table 1 threshold other than
// Sauvola and Niblack: FP32 threshold, and in MODE_FP64 the certified bound
// (undecided pixels go to the out-of-line FP64 decision); in MODE_REPORT the
// FP32-vs-FP64 flips and the largest |t32 - t64|.
// In MODE_REPORT also the largest ratio |t32 - t64| / bound over the two
// variance roundings the kernels use, (V / n) / n here and V (1 / n^2) on the
// pipelined path, each with its own certified bound: below 1 means that
// every FP32 decision the FP64 mode keeps equals the canonical FP64 one.
template <int METHOD, int MODE, bool INTERIOR, typename S2T>
__device__ __forceinline__ void ext_row8(const ExtF &F, const ThreshExt &T, const Global &G, uint2 P,
                                         uint32_t off1, const uint32_t (&p1)[kColsPerLane], S2T off2,
                                         const S2T (&p2)[kColsPerLane], uint32_t nw, uint32_t nrow,
                                         const uint32_t (&cols)[kColsPerLane], float inv_nw,
                                         float inv_rows, const float (&inv_cols)[kColsPerLane],
                                         int64_t j0, int64_t W, uint32_t &byte, uint32_t &undecided,
                                         unsigned long long &nflip, double &maxdt, double &maxratio)
{
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        const uint32_t S1 = off1 + p1[m];
        const uint64_t S2 = (uint64_t)(off2 + p2[m]);
        const uint32_t n = INTERIOR ? nw : nrow * cols[m];
        const float inv_n = INTERIOR ? inv_nw : inv_rows * inv_cols[m];
        const float mu = __uint2float_rn(S1) * inv_n;
        const float var = (v_float<S2T>(n, S2, S1) * inv_n) * inv_n;
        float bnd;
        const float t = ext_t32<METHOD>(F, mu, var, inv_n, bnd);
        const float d = t - pixel_f(P, m);
        const uint32_t bit = __float_as_uint(d) >> 31;
        byte |= bit << m;
        if (MODE == MODE_FP64) {
            undecided |= (fabsf(d) <= bnd ? 1u : 0u) << m;
        } else if (MODE == MODE_REPORT) {
            if (j0 + m < W) {
                const double t64 = canonical_t_ext(METHOD, S1, S2, n, T.k, T.R, T.X, G);
                const uint32_t b64 = ((double)byte_at(P, m) <= t64) ? 0u : 1u;
                nflip += (b64 != bit);
                const double dt = fabs((double)t - t64);
                maxdt = dt > maxdt ? dt : maxdt;
                const float varB = v_float<S2T>(n, S2, S1) * (inv_n * inv_n);
                float bndB;
                const float tB = ext_t32<METHOD>(F, mu, varB, inv_n, bndB);
                const double ra = dt / (double)bnd, rb = fabs((double)tB - t64) / (double)bndB;
                maxratio = fmax(maxratio, fmax(ra, rb));
            }
        }
    }
}

// Warm-up from stripe sums: `st` holds (C, D) = (sum I, sum I^2) of every
// column over the window rows of this tile's first row (the stripe
// pre-pass), so E_j = C_{j+r} - C_{j-l} directly and the anchor is the sum of
// C and D over the anchor columns [ac0, aend).  Columns outside [0, W) are 0.
__device__ __forceinline__ void warm_from_stripes(const uint2 *st, int64_t W, int64_t colA,
                                                  int64_t colB, int64_t ac0, int64_t aend, int lane,
                                                  int32_t *E1, uint32_t *E2, uint32_t &a1p,
                                                  uint32_t &a2p)
{
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        const int64_t xa = colA + m, xb = colB + m;
        const uint2 ca = (xa >= 0 && xa < W && BZ_DBG_IN(st + xa, 8, st, (size_t)W * 8, kDbgScratch))
                             ? __ldg(st + xa)
                             : make_uint2(0u, 0u);
        const uint2 cb = (xb >= 0 && xb < W && BZ_DBG_IN(st + xb, 8, st, (size_t)W * 8, kDbgScratch))
                             ? __ldg(st + xb)
                             : make_uint2(0u, 0u);
        E1[m] = (int32_t)(ca.x - cb.x);
        E2[m] = ca.y - cb.y;
    }
    for (int64_t x = ac0 + lane; x < aend; x += 32) {
        if (x >= 0 && x < W && BZ_DBG_IN(st + x, 8, st, (size_t)W * 8, kDbgScratch)) {
            const uint2 c = __ldg(st + x);
            a1p += c.x;
            a2p += c.y;
        }
    }
}

// S2T: uint32_t when h*w <= 66051 (S2 < 2^32), else unsigned long long.
// EXT: the Table 1 thresholds other than Sauvola and Niblack (T.method).
// INTERIOR: every lane's byte streams and outputs lie inside the row, the
// image and pitch allow aligned 8-byte loads, and every output column has
// the full window width w (warp-uniform; decided by window_tile).
template <int MODE, bool VEC, bool INTERIOR, typename S2T, bool EXT = false, bool WARMB = false>
__device__ __forceinline__ void window_rows(const Image &g, const Window &win, const Thresh &T,
                                            const Outputs &o, int64_t x0, int64_t y0, int64_t y1,
                                            int lane, const uint2 *stripe = nullptr)
{
    const int64_t W = g.W, H = g.H;
    const int64_t j0 = x0 + (int64_t)kColsPerLane * lane;
    const int l = win.l, r = win.r, oo = win.o, u = win.u;
    [[maybe_unused]] const size_t img_ext = dbg_image_extent(g);

    const int64_t colA = j0 + r, colB = j0 - l;
    const bool fastA = INTERIOR || (VEC && colA >= 0 && colA + 8 <= W);
    const bool fastB = INTERIOR || (VEC && colB >= 0 && colB + 8 <= W);
    const bool fastP = INTERIOR || (VEC && j0 + 8 <= W);
    const int kA = (int)(colA & 7), kB = (int)(colB & 7);  // warp-uniform
    const unsigned selA = (unsigned)(kA & 3) * 0x1111u + 0x3210u;
    const unsigned selB = (unsigned)(kB & 3) * 0x1111u + 0x3210u;

    auto load_row = [&](int64_t row, uint2 &A, uint2 &B) {
        const uint8_t *rp = g.img + row * g.pitch;
        if (INTERIOR) {
            A = ld8_fast(rp + colA, kA, selA, g.img, img_ext);
            B = ld8_fast(rp + colB, kB, selB, g.img, img_ext);
        } else {
            A = ld8<VEC>(rp, colA, fastA, kA, selA, W, g.img, img_ext);
            B = ld8<VEC>(rp, colB, fastB, kB, selB, W, g.img, img_ext);
        }
    };

    // per-column clipped widths (edge tiles only)
    uint32_t cols[kColsPerLane];
    float inv_cols[kColsPerLane];
    if (!INTERIOR) {
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            const int64_t j = j0 + m;
            const int64_t hi = j + r < W - 1 ? j + r : W - 1;
            const int64_t lo = j - l > -1 ? j - l : -1;
            const int64_t c = hi - lo;
            cols[m] = (uint32_t)(c < 1 ? 1 : c);  // c < 1 only for j >= W
            inv_cols[m] = __frcp_rn((float)cols[m]);
        }
    }
    const float inv_w = __frcp_rn((float)win.w);
    const float inv_h = __frcp_rn((float)win.h);
    const float inv_hw = inv_h * inv_w;

    // anchor window: columns [x0-l, x0-1+r] (the window of column x0-1)
    const int64_t ac0 = x0 - l, aend = x0 + r;
    const int64_t a4 = ac0 >= 0 ? (ac0 & ~(int64_t)3) : -((-ac0 + 3) & ~(int64_t)3);
    // one word per lane covers the anchor when it spans at most 32 words
    const bool one_word = INTERIOR && (aend - a4) <= 128;
    const int64_t c4 = a4 + 4 * lane;
    const bool has_word = c4 < aend;
    uint32_t keep = 0xFFFFFFFFu;
    if (c4 < ac0)
        keep &= 0xFFFFFFFFu << (8 * (int)(ac0 - c4));
    if (c4 + 4 > aend)
        keep = (c4 >= aend) ? 0u : (keep & (0xFFFFFFFFu >> (8 * (int)(c4 + 4 - aend))));
    // interior anchors wider than 32 words: up to 5 words per lane (w <= 511)
    // with their masks fixed for the whole tile
    constexpr int kAW = 5;
    uint32_t keepk[kAW];
#pragma unroll
    for (int k = 0; k < kAW; k++) {
        const int64_t ck = c4 + 128 * k;
        uint32_t m = 0xFFFFFFFFu;
        if (ck < ac0)
            m &= 0xFFFFFFFFu << (8 * (int)(ac0 - ck));
        if (ck + 4 > aend)
            m = (ck >= aend) ? 0u : (m & (0xFFFFFFFFu >> (8 * (int)(ck + 4 - aend))));
        keepk[k] = m;
    }
    auto anchor_row = [&](int64_t row, uint32_t &s1, uint32_t &s2) {
        const uint8_t *rp = g.img + row * g.pitch;
        if (one_word) {
            if (has_word) {
                const uint32_t wd = (BZ_DBG_IN(rp + c4, 4, g.img, img_ext, kDbgImage)
                                         ? __ldg(reinterpret_cast<const uint32_t *>(rp + c4))
                                         : 0u) &
                                    keep;
                s1 = __dp4a(wd, 0x01010101u, s1);
                s2 = __dp4a(wd, wd, s2);
            }
        } else if (INTERIOR) {
            // every word lies inside the row (the tile is interior), so only
            // the words past the anchor are skipped
#pragma unroll
            for (int k = 0; k < kAW; k++) {
                if (c4 + 128 * k < aend) {
                    const uint32_t wd =
                        (BZ_DBG_IN(rp + c4 + 128 * k, 4, g.img, img_ext, kDbgImage)
                             ? __ldg(reinterpret_cast<const uint32_t *>(rp + c4 + 128 * k))
                             : 0u) &
                        keepk[k];
                    s1 = __dp4a(wd, 0x01010101u, s1);
                    s2 = __dp4a(wd, wd, s2);
                }
            }
        } else {
            anchor_words<VEC>(rp, a4, ac0, aend, W, lane, s1, s2, g.img, img_ext);
        }
    };

    // ---- warm-up: E and the anchor for row y0 (window rows (y0-o, y0+u])
    int32_t E1[kColsPerLane];
    uint32_t E2[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        E1[m] = 0;
        E2[m] = 0;
    }
    uint32_t a1p = 0, a2p = 0;
    if (stripe) {
        warm_from_stripes(stripe, W, colA, colB, ac0, aend, lane, E1, E2, a1p, a2p);
    } else {
        int64_t a_lo = y0 - oo + 1, a_hi = y0 + u;
        if (a_lo < 0)
            a_lo = 0;
        if (a_hi > H - 1)
            a_hi = H - 1;
        const uint2 Z = make_uint2(0u, 0u);
        if (WARMB) {
            // latency-bound launches (few, short tiles): the loads of
            // kWarmRows rows are issued before any is accumulated
            for (int64_t a = a_lo; a <= a_hi; a += kWarmRows) {
                uint2 Ar[kWarmRows], Br[kWarmRows];
                uint32_t w1r[kWarmRows], w2r[kWarmRows];
#pragma unroll
                for (int q = 0; q < kWarmRows; q++) {
                    Ar[q] = Br[q] = Z;
                    w1r[q] = w2r[q] = 0u;
                    if (a + q <= a_hi) {  // warp-uniform
                        load_row(a + q, Ar[q], Br[q]);
                        anchor_row(a + q, w1r[q], w2r[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < kWarmRows; q += 4) {  // rows past a_hi are zero
                    const uint2 A4[4] = {Ar[q], Ar[q + 1], Ar[q + 2], Ar[q + 3]};
                    const uint2 B4[4] = {Br[q], Br[q + 1], Br[q + 2], Br[q + 3]};
                    warm8x4(A4, B4, E1, E2);
                }
#pragma unroll
                for (int q = 0; q < kWarmRows; q++) {
                    a1p += w1r[q];
                    a2p += w2r[q];
                }
            }
            a_hi = a_lo - 1;  // done: skip the loops below
        }
        // four rows at a time (their loads issued together)
        for (; a_lo + 3 <= a_hi; a_lo += 4) {
            uint2 Ar[4], Br[4];
            uint32_t w1r[4], w2r[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                load_row(a_lo + q, Ar[q], Br[q]);
                w1r[q] = w2r[q] = 0u;
                anchor_row(a_lo + q, w1r[q], w2r[q]);
            }
            warm8x4(Ar, Br, E1, E2);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                a1p += w1r[q];
                a2p += w2r[q];
            }
        }
        // the rest with one row of look-ahead: the loads of row a+1 are in
        // flight while row a is accumulated
        uint2 A = Z, B = Z;
        uint32_t w1 = 0, w2 = 0;
        if (a_lo <= a_hi) {
            load_row(a_lo, A, B);
            anchor_row(a_lo, w1, w2);
        }
        for (int64_t a = a_lo; a <= a_hi; a++) {
            uint2 An = Z, Bn = Z;
            uint32_t v1 = 0, v2 = 0;
            if (a < a_hi) {
                load_row(a + 1, An, Bn);
                anchor_row(a + 1, v1, v2);
            }
            warm8(A, B, E1, E2);
            a1p += w1;
            a2p += w2;
            A = An;
            B = Bn;
            w1 = v1;
            w2 = v2;
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
    double maxdt = 0.0, maxratio = 0.0;

    uint2 nA = make_uint2(0, 0), nB = nA, nC = nA, nD = nA, nP = nA;
    uint32_t nd1 = 0, nd2 = 0;
    auto load_centre = [&](int64_t i) {
        const uint8_t *prow = g.img + i * g.pitch;
        if (INTERIOR && !BZ_DBG_IN(prow + j0, 8, g.img, img_ext, kDbgImage))
            return make_uint2(0u, 0u);
        return INTERIOR ? __ldg(reinterpret_cast<const uint2 *>(prow + j0))
                        : ld8<VEC>(prow, j0, fastP, 0, 0x3210u, W, g.img, img_ext);
    };
    auto prefetch = [&](int64_t i) {
        const int64_t ra = i + u, rb = i - oo;
        nA = nB = nC = nD = make_uint2(0, 0);
        if (MODE != MODE_SUMS)
            nP = load_centre(i);
        uint32_t e1 = 0, e2 = 0, x1 = 0, x2 = 0;
        if (ra < H) {
            load_row(ra, nA, nB);
            anchor_row(ra, e1, e2);
        }
        if (rb >= 0) {
            load_row(rb, nC, nD);
            anchor_row(rb, x1, x2);
        }
        nd1 = e1 - x1;
        nd2 = e2 - x2;
    };
    uint2 P = MODE != MODE_SUMS ? load_centre(y0) : make_uint2(0u, 0u);
    if (y0 + 1 < y1)
        prefetch(y0 + 1);

    const bool simple = !EXT && T.method == 0 && T.alpha >= 0.0f && T.beta >= 0.0f;  // Sauvola, 0<=k<=1
    Global G{};
    ExtF F{};
    // only instantiated with EXT for a ThreshExt argument (k_window_ext)
    const ThreshExt &TX = static_cast<const ThreshExt &>(T);
    if (EXT) {
        G = global_lms(*TX.gs, TX.N);
        F = make_extf(T.method, T.k, T.R, TX.X, G, T.eps);
    }

    for (int64_t i = y0; i < y1; i++) {
        if (i > y0) {
            P = nP;
            slide8(nA, nB, nC, nD, E1, E2);
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
            run2 += (S2T)(int64_t)(int32_t)E2[m];
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
                        if (BZ_DBG_IN(o.S1 + idx, 4, o.S1, (size_t)o.sums_n * 4, kDbgOutput))
                            o.S1[idx] = off1 + p1[m];
                    if (o.S2)
                        if (BZ_DBG_IN(o.S2 + idx, 8, o.S2, (size_t)o.sums_n * 8, kDbgOutput))
                            o.S2[idx] = (uint64_t)(off2 + p2[m]);
                    if (o.n)
                        if (BZ_DBG_IN(o.n + idx, 4, o.n, (size_t)o.sums_n * 4, kDbgOutput))
                            o.n[idx] = nrow * (INTERIOR ? (uint32_t)win.w : cols[m]);
                }
            }
            continue;
        }

        const bool full_rows = nrow == (uint32_t)win.h;  // warp-uniform
        const float inv_rows = full_rows ? inv_h : __frcp_rn((float)rows);
        uint32_t byte = 0, undecided = 0;
        const uint32_t nw = nrow * (uint32_t)win.w;
        const float inv_nw = full_rows ? inv_hw : inv_rows * inv_w;
        if (MODE == MODE_FP64_DIRECT) {
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const uint32_t n = INTERIOR ? nw : nrow * cols[m];
                byte |= (EXT ? fp64_bit_ext(T.method, (uint32_t)byte_at(P, m), off1 + p1[m],
                                            (uint64_t)(off2 + p2[m]), n, T.k, T.R, TX.X.alpha1,
                                            TX.X.k1, TX.X.k2, TX.X.gamma, TX.X.p, TX.X.q, G.L, G.M, G.S)
                             : fp64_bit(T.method, (uint32_t)byte_at(P, m), off1 + p1[m],
                                        (uint64_t)(off2 + p2[m]), n, T.k, T.R))
                        << m;
            }
        } else if (EXT) {
#define BZ_EXT_ROW(M_)                                                                             \
    ext_row8<M_, MODE, INTERIOR, S2T>(F, TX, G, P, off1, p1, off2, p2, nw, nrow, cols, inv_nw, inv_rows, \
                                      inv_cols, j0, W, byte, undecided, nflip, maxdt, maxratio)
            switch (T.method) {
            case METHOD_WOLF: BZ_EXT_ROW(METHOD_WOLF); break;
            case METHOD_FENG: BZ_EXT_ROW(METHOD_FENG); break;
            case METHOD_RAIS: BZ_EXT_ROW(METHOD_RAIS); break;
            case METHOD_NICK: BZ_EXT_ROW(METHOD_NICK); break;
            default: BZ_EXT_ROW(METHOD_PHANSALKAR); break;
            }
#undef BZ_EXT_ROW
        } else if (INTERIOR && simple && MODE != MODE_REPORT) {
            // Sauvola with 0 <= k <= 1: t = m (alpha + beta s), |terms| = t
            const float inv_n2 = inv_nw * inv_nw;
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const uint32_t S1 = off1 + p1[m];
                const float mu = __uint2float_rn(S1) * inv_nw;
                const float var = v_float<S2T>(nw, (uint64_t)(off2 + p2[m]), S1) * inv_n2;
                const float t = mu * fmaf(T.beta, sqrt_approx(var), T.alpha);
                const float d = t - pixel_f(P, m);  // d < 0  <=>  I > t
                byte |= (__float_as_uint(d) >> 31) << m;
                if (MODE == MODE_FP64)
                    undecided |= (fabsf(d) <= fmaf(T.eps, t, T.delta64) ? 1u : 0u) << m;
            }
        } else {
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                const uint32_t S1 = off1 + p1[m];
                const uint64_t S2 = (uint64_t)(off2 + p2[m]);
                const uint32_t n = INTERIOR ? nw : nrow * cols[m];
                const float inv_n = INTERIOR ? inv_nw : inv_rows * inv_cols[m];
                const float mu = __uint2float_rn(S1) * inv_n;
                const float var = (v_float<S2T>(n, S2, S1) * inv_n) * inv_n;
                const float s = sqrt_approx(var);
                const float t = fmaf(fmaf(T.beta, mu, T.gamma), s, T.alpha * mu);
                const float d = t - pixel_f(P, m);
                const uint32_t bit = __float_as_uint(d) >> 31;
                byte |= bit << m;
                if (MODE == MODE_FP64) {
                    const float mag = fmaf(fmaf(T.abeta, mu, T.agamma), s, T.aalpha * mu);
                    undecided |= (fabsf(d) <= fmaf(T.eps, mag, T.delta64) ? 1u : 0u) << m;
                } else if (MODE == MODE_REPORT) {
                    if (j0 + m < W) {
                        const double t64 = canonical_t(T.method, S1, S2, n, T.k, T.R);
                        const uint32_t I = (uint32_t)byte_at(P, m);
                        const uint32_t b64 = ((double)I <= t64) ? 0u : 1u;
                        // the FP32 value of the path this pixel takes in
                        // BZ_FP32 (t here is the generic form's)
                        double t32 = (double)t;
                        if (o.report_path == kReportSmall) {
                            const float inv1 = __frcp_rn((float)n);
                            const float mu1 = __uint2float_rn(S1) * inv1;
                            const float s1 = sqrt_approx((v_float<S2T>(n, S2, S1) * inv1) * inv1);
                            t32 = (double)fmaf(fmaf(T.beta, mu1, T.gamma), s1, T.alpha * mu1);
                        } else if (o.report_path == kReportPipe && INTERIOR) {
                            const float an = T.alpha * inv_n, gn = T.gamma * inv_n, bn2 = (T.beta * inv_n) * inv_n;
                            const float S1f = __uint2float_rn(S1);
                            const float sq = sqrt_approx(__ull2float_rn((uint64_t)n * S2 - (uint64_t)S1 * (uint64_t)S1));
                            const float If = pixel_f(P, m);
                            const float dP = simple ? fmaf(S1f, fmaf(bn2, sq, an), -If)
                                                    : fmaf(fmaf(bn2, S1f, gn), sq, fmaf(S1f, an, -If));
                            t32 = (double)dP + (double)I;
                        } else if (o.report_path == kReportPipe || (INTERIOR && simple)) {
                            const float sB = sqrt_approx(v_float<S2T>(n, S2, S1) * (inv_n * inv_n));
                            t32 = simple ? (double)(mu * fmaf(T.beta, sB, T.alpha))
                                         : (double)fmaf(fmaf(T.beta, mu, T.gamma), sB, T.alpha * mu);
                        }
                        const uint32_t b32 = t32 < (double)I ? 1u : 0u;
                        nflip += (b64 != b32);
                        const double dt = fabs(t32 - t64);
                        maxdt = dt > maxdt ? dt : maxdt;
                        // the certified bound of every evaluation form the FP64
                        // mode uses: general t with var = (V / n) / n (this
                        // routine) and var = V (1 / n^2) (pipelined path), and
                        // the Sauvola form m (alpha + beta s) with the latter
                        const float magA = fmaf(fmaf(T.abeta, mu, T.agamma), s, T.aalpha * mu);
                        const double rA = dt / (double)fmaf(T.eps, magA, T.delta64);
                        const float sB = sqrt_approx(v_float<S2T>(n, S2, S1) * (inv_n * inv_n));
                        const float tB = fmaf(fmaf(T.beta, mu, T.gamma), sB, T.alpha * mu);
                        const float magB = fmaf(fmaf(T.abeta, mu, T.agamma), sB, T.aalpha * mu);
                        const double rB = fabs((double)tB - t64) / (double)fmaf(T.eps, magB, T.delta64);
                        double rS = 0.0;
                        if (simple) {
                            const float tS = mu * fmaf(T.beta, sB, T.alpha);
                            rS = fabs((double)tS - t64) / (double)fmaf(T.eps, tS, T.delta64);
                        }
                        // the interior pipelined form: d = t - I from row
                        // constants, against the launch constant T.bnd_c
                        const float an = T.alpha * inv_n, gn = T.gamma * inv_n, bn2 = (T.beta * inv_n) * inv_n;
                        const float S1f = __uint2float_rn(S1);
                        const float sqN = sqrt_approx(
                            __ull2float_rn((uint64_t)n * S2 - (uint64_t)S1 * (uint64_t)S1));
                        const float If = pixel_f(P, m);
                        const float dN = simple ? fmaf(S1f, fmaf(bn2, sqN, an), -If)
                                                : fmaf(fmaf(bn2, S1f, gn), sqN, fmaf(S1f, an, -If));
                        const double rN = fabs((double)dN - (t64 - (double)I)) / (double)T.bnd_c;
                        maxratio = fmax(maxratio, fmax(fmax(rA, rN), fmax(rB, rS)));
                    }
                }
            }
        }
        if (MODE == MODE_FP64) {
            // near-ties: canonical FP64 evaluation, off the hot path
            if (!INTERIOR && j0 + 8 > W)
                undecided &= (1u << (j0 < W ? W - j0 : 0)) - 1u;
            if (__any_sync(0xFFFFFFFFu, undecided != 0) && undecided) {
#pragma unroll
                for (int m = 0; m < kColsPerLane; m++) {
                    if (undecided >> m & 1u) {
                        const uint32_t n = INTERIOR ? nw : nrow * cols[m];
                        const uint32_t b =
                            EXT ? fp64_bit_ext(T.method, (uint32_t)byte_at(P, m), off1 + p1[m],
                                               (uint64_t)(off2 + p2[m]), n, T.k, T.R, TX.X.alpha1,
                                               TX.X.k1, TX.X.k2, TX.X.gamma, TX.X.p, TX.X.q, G.L, G.M,
                                               G.S)
                                : fp64_bit(T.method, (uint32_t)byte_at(P, m), off1 + p1[m],
                                           (uint64_t)(off2 + p2[m]), n, T.k, T.R);
                        byte = (byte & ~(1u << m)) | (b << m);
                    }
                }
                nfb += __popc(undecided);
            }
        }
        if (MODE != MODE_REPORT && j0 < W) {
            if (!INTERIOR && j0 + 8 > W)
                byte &= (1u << (W - j0)) - 1u;  // padding bits are 0
            uint8_t *dst = o.bits + (i - o.out_row0) * o.out_pitch + ((j0 >> 3) - o.out_byte0);
            if (BZ_DBG_IN(dst, 1, o.bits, o.bits_bytes, kDbgOutput))
                *dst = (uint8_t)byte;
        }
    }

    if (MODE == MODE_FP64 && o.fallbacks) {
        const unsigned v = __reduce_add_sync(0xFFFFFFFFu, (unsigned)nfb);
        if (lane == 0 && v)
            atomicAdd(o.fallbacks, (unsigned long long)v);
    }
    if (MODE == MODE_REPORT) {
        unsigned long long v = nflip;
        double mx = maxdt, mr = maxratio;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
            const double y = __shfl_xor_sync(0xFFFFFFFFu, mx, d);
            mx = y > mx ? y : mx;
            const double z = __shfl_xor_sync(0xFFFFFFFFu, mr, d);
            mr = z > mr ? z : mr;
        }
        if (lane == 0) {
            if (v && o.flips)
                atomicAdd(o.flips, v);
            if (o.maxdt_bits)
                atomicMax(o.maxdt_bits, (unsigned long long)__double_as_longlong(mx));
            if (o.maxratio_bits)
                atomicMax(o.maxratio_bits, (unsigned long long)__double_as_longlong(mr));
        }
    }
}

// Edge tiles: a byte stream that starts at column c outside [0, W - 8] is
// read from the nearest in-row 8 bytes, at cl = clamp(c, 0, W - 8), and
// shifted by sh = cl - c bytes (clamped to +-8), so that byte m holds column
// c + m and columns outside [0, W) read as 0.  Needs W >= 8.
__device__ __forceinline__ void edge_clamp(int64_t c, int64_t W, int64_t &cl, int &sh)
{
    cl = c < 0 ? 0 : (c > W - 8 ? W - 8 : c);
    const int64_t d = cl - c;
    sh = d > 8 ? 8 : (d < -8 ? -8 : (int)d);
}

__device__ __forceinline__ uint2 shift8(uint2 v, int sh)
{
    unsigned long long x = ((unsigned long long)v.y << 32) | v.x;
    const unsigned b = 8u * (unsigned)(sh < 0 ? -sh : sh);
    x = b >= 64u ? 0ull : (sh > 0 ? x << b : x >> b);
    return make_uint2((uint32_t)x, (uint32_t)(x >> 32));
}

// Column sums over four rows of one word (columns c .. c+3): the bytes of each
// column are gathered into one word (4 x 4 byte transpose), then one DP4A adds
// the column's sum and one its sum of squares.
__device__ __forceinline__ void col4_sums(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t *C,
                                          uint32_t *D)
{
    const uint32_t lo01 = __byte_perm(r0, r1, 0x5140u), hi01 = __byte_perm(r0, r1, 0x7362u);
    const uint32_t lo23 = __byte_perm(r2, r3, 0x5140u), hi23 = __byte_perm(r2, r3, 0x7362u);
    const uint32_t c[4] = {__byte_perm(lo01, lo23, 0x5410u), __byte_perm(lo01, lo23, 0x7632u),
                           __byte_perm(hi01, hi23, 0x5410u), __byte_perm(hi01, hi23, 0x7632u)};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        C[k] = __dp4a(c[k], 0x01010101u, C[k]);
        D[k] = __dp4a(c[k], c[k], D[k]);
    }
}

// Warm-up of the pipelined path (row y0, window rows a_lo .. a_hi) as column
// sums (Sec. 3.1 stripe identity): every lane sums its own 8 columns (one
// aligned 8-byte load per row) and AW words of the halo, the columns
// [x0 - 64 AW, x0) and [x0 + 256, x0 + 256 + r) that the window edges of the
// tile reach (l, r <= 64 AW).  The sums C, D then go through the warp's shared
// memory once, E_j = C_{j+r} - C_{j-l} (likewise for the squares), and the
// anchor is the sum of C and D over the columns [x0 - l, x0 + r).  The same
// integers as sliding both window-edge streams down the rows (E-form), with
// one load stream instead of two plus the anchor's.  EDGE: columns outside
// [0, W) count as 0 (words left of column 0 or starting at W or later are not
// read; the sums of columns >= W, read from the row's padding, are cleared).
// `sm`: the warp's shared memory, 4608 bytes used (column k of
// [x0 - 64 AW, x0 + 256 + 64 AW) at word k + k / 8, so that lanes 8 columns
// apart read distinct banks); free again when this returns.
template <int AW, bool EDGE>
__device__ __forceinline__ void warm_cols(const Image &g, const Window &win, int64_t x0, int lane,
                                          int64_t a_lo, int64_t a_hi, uint32_t *sm, int32_t *E1,
                                          uint32_t *E2, uint32_t &a1p, uint32_t &a2p)
{
    constexpr int HALO = 64 * AW;
    constexpr int NPH = (kTileCols + 2 * HALO) * 9 / 8;  // words per array
    [[maybe_unused]] const size_t ext = dbg_image_extent(g);
    const int l = win.l, r = win.r;
    const int64_t j0 = x0 + kColsPerLane * lane;
    // halo word q of this lane: AW = 1, lanes 0-15 left and 16-31 right; AW =
    // 2, word 0 left and word 1 right.  `hk`: its first column, relative to
    // x0 - HALO.  Right words past the window's reach are not read.
    int hk[AW];
    bool hv[AW];
#pragma unroll
    for (int q = 0; q < AW; q++) {
        const bool left = AW == 1 ? lane < 16 : q == 0;
        const int k = AW == 1 ? 4 * (lane & 15) : 4 * lane;
        hk[q] = left ? k : HALO + kTileCols + k;
        hv[q] = left || k < r;
        if (EDGE) {
            const int64_t c = x0 - HALO + hk[q];
            hv[q] = hv[q] && c >= 0 && c < g.W;
        }
    }
    const bool ov = !EDGE || j0 < g.W;
    uint32_t Co[kColsPerLane], Do[kColsPerLane], Ch[AW][4], Dh[AW][4];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++)
        Co[m] = Do[m] = 0u;
#pragma unroll
    for (int q = 0; q < AW; q++)
#pragma unroll
        for (int k = 0; k < 4; k++)
            Ch[q][k] = Dh[q][k] = 0u;

    const uint8_t *po = g.img + j0;
    const uint8_t *ph[AW];
#pragma unroll
    for (int q = 0; q < AW; q++)
        ph[q] = g.img + (x0 - HALO + hk[q]);
    // four rows per round; rows past a_hi read as zero (the last round only)
    auto group = [&](int64_t a, bool partial) {
        uint2 O[4];
        uint32_t Hw[AW][4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            O[q] = make_uint2(0u, 0u);
#pragma unroll
            for (int w = 0; w < AW; w++)
                Hw[w][q] = 0u;
            if (!partial || a + q <= a_hi) {  // warp-uniform
                const int64_t ro = (a + q) * g.pitch;
                if (ov && BZ_DBG_IN(po + ro, 8, g.img, ext, kDbgImage))
                    O[q] = __ldg(reinterpret_cast<const uint2 *>(po + ro));
#pragma unroll
                for (int w = 0; w < AW; w++)
                    if (hv[w] && BZ_DBG_IN(ph[w] + ro, 4, g.img, ext, kDbgImage))
                        Hw[w][q] = __ldg(reinterpret_cast<const uint32_t *>(ph[w] + ro));
            }
        }
        col4_sums(O[0].x, O[1].x, O[2].x, O[3].x, Co, Do);
        col4_sums(O[0].y, O[1].y, O[2].y, O[3].y, Co + 4, Do + 4);
#pragma unroll
        for (int w = 0; w < AW; w++)
            col4_sums(Hw[w][0], Hw[w][1], Hw[w][2], Hw[w][3], Ch[w], Dh[w]);
    };
    int64_t a = a_lo;
    for (; a + 3 <= a_hi; a += 4)
        group(a, false);
    if (a <= a_hi)
        group(a, true);
    if (EDGE) {  // columns >= W were read from the row padding
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++)
            if (j0 + m >= g.W)
                Co[m] = Do[m] = 0u;
#pragma unroll
        for (int q = 0; q < AW; q++)
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (x0 - HALO + hk[q] + k >= g.W)
                    Ch[q][k] = Dh[q][k] = 0u;
    }

    // the anchor: own columns below x0 + r, left-halo columns from x0 - l
    const int own_n = r - kColsPerLane * lane;  // own columns inside the anchor
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++)
        if (m < own_n) {
            a1p += Co[m];
            a2p += Do[m];
        }
#pragma unroll
    for (int q = 0; q < AW; q++)
        if (hk[q] < HALO)
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (hk[q] + k >= HALO - l) {
                    a1p += Ch[q][k];
                    a2p += Dh[q][k];
                }

    uint32_t *sC = sm, *sD = sm + NPH;
    __syncwarp();  // the previous tile's last row may still read the slots
    {
        const int p0 = HALO + HALO / 8 + 9 * lane;  // own column 0 (HALO + 8 lane)
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            sC[p0 + m] = Co[m];
            sD[p0 + m] = Do[m];
        }
#pragma unroll
        for (int q = 0; q < AW; q++) {
            // hk a multiple of 4: its 4 columns share one pad word; words not
            // read are zero columns
            const int p = hk[q] + (hk[q] >> 3);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                sC[p + k] = Ch[q][k];
                sD[p + k] = Dh[q][k];
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        const int iA = HALO + kColsPerLane * lane + m + r, iB = HALO + kColsPerLane * lane + m - l;
        const int pA = iA + (iA >> 3), pB = iB + (iB >> 3);
        E1[m] = (int32_t)(sC[pA] - sC[pB]);
        E2[m] = sD[pA] - sD[pB];
    }
    __syncwarp();  // the slots are rewritten next
}

// Per-row constants of the pipelined path's threshold (a 32-row table in the
// warp's shared memory): the clipped row count, n = rows * w, 1/n from
// correctly rounded reciprocals (edge tiles: 1/rows, the column factor comes
// from the column table), the interior form's alpha/n, gamma/n and beta/n^2,
// and the output row's offset.
struct RowC {
    float inv_nw, an, gn, bn2;
    uint32_t nrow, nw;
    int64_t dst;
};

// FP32 d = t - I of the interior form: S1 (alpha/n + beta/n^2 sqrt(V)) - I
// (SIMPLE: Sauvola with alpha, beta >= 0), else alpha S1/n + (beta S1/n^2 +
// gamma/n) sqrt(V) - I, with S1 and V = n S2 - S1^2 each rounded once (V32:
// V below 2^32, exact in wrapping 32-bit products); certified when |d| >
// bnd_c.
__device__ __forceinline__ float eval_interior(bool SIMPLE, bool V32, uint32_t S1, uint32_t S2, uint32_t nw,
                                               float an, float gn, float bn2, float If)
{
    const float S1f = __uint2float_rn(S1);
    const float Vf = V32 ? __uint2float_rn(nw * S2 - S1 * S1) : __ull2float_rn((uint64_t)nw * S2 - (uint64_t)S1 * S1);
    const float sq = sqrt_approx(Vf);
    return SIMPLE ? fmaf(S1f, fmaf(bn2, sq, an), -If) : fmaf(fmaf(bn2, S1f, gn), sq, fmaf(S1f, an, -If));
}

// FP32 threshold of one pixel from m = S1/n and var = V/n^2 with its
// per-pixel certified bound: returns the bit and sets slack = |t - I| -
// bound, certified when > 0.  SIMPLE: Sauvola with alpha, beta >= 0.
template <int EXTM, typename S2T>
__device__ __forceinline__ uint32_t eval_bounded(const Thresh &T, const ExtF &F, bool SIMPLE, uint32_t n_m,
                                                 float inv_m, uint32_t S1, uint32_t S2, float If, float &slack)
{
    const float mu = __uint2float_rn(S1) * inv_m;
    const float var = v_float<S2T>(n_m, (uint64_t)S2, S1) * (inv_m * inv_m);
    float t, bnd;
    if (EXTM) {
        t = ext_t32<EXTM ? EXTM : METHOD_WOLF>(F, mu, var, inv_m, bnd);
    } else if (SIMPLE) {
        t = mu * fmaf(T.beta, sqrt_approx(var), T.alpha);
        bnd = fmaf(T.eps, t, T.delta64);
    } else {
        const float s = sqrt_approx(var);
        t = fmaf(fmaf(T.beta, mu, T.gamma), s, T.alpha * mu);
        bnd = fmaf(T.eps, fmaf(fmaf(T.abeta, mu, T.agamma), s, T.aalpha * mu), T.delta64);
    }
    const float d = t - If;
    slack = fabsf(d) - bnd;
    return __float_as_uint(d) >> 31;
}

// The near-tie path of one row of the pipelined kernel (BZ_FP64), called by
// the whole warp when some lane has an uncertified pixel.  Out of line, so
// that its registers do not weigh on the row loop's allocation (inline, it
// cost the loop ~4 % of its time with no near-tie taken).  The lanes with an
// uncertified pixel re-read the row's sums from the slot `par` and
// re-evaluate their 8 pixels in the same FP32 form as the row loop; the
// uncertified ones are then decided in FP64, spread over the lanes of the
// warp (up to 32 per round), since FP64 is slow on this part and such pixels
// come in clusters (flat or saturated areas).  Returns the lane's byte in
// bits 0-7 and its number of FP64 decisions above.
template <bool EDGE, int EXTM, typename TT>
static __device__ __noinline__ uint32_t near_tie_row(const TT T, const ExtF F, uint4 *slots, int par, int lane,
                                                     uint2 P, uint32_t byte, bool need, const RowC rc,
                                                     bool simple, uint32_t vmask)
{
    const uint4 *sl = slots + par * 128;
    const uint2 *ctab = reinterpret_cast<const uint2 *>(slots + 256);
    auto count_of = [&](int ln, int m, uint32_t &n_m, float &inv_m) {
        if (EDGE) {
            const uint2 e = ctab[m * 32 + ln];
            n_m = rc.nrow * e.y;
            inv_m = rc.inv_nw * __uint_as_float(e.x);
        } else {
            n_m = rc.nw;
            inv_m = rc.inv_nw;
        }
    };
    __syncwarp();  // the slot and the column table are read across lanes
    const volatile uint32_t *vs = reinterpret_cast<const volatile uint32_t *>(sl);
    uint32_t und = 0;
    if (need) {
        byte = 0;
        for (int m = 0; m < kColsPerLane; m++) {
            const uint32_t S1 = vs[((m >> 2) * 32 + lane) * 4 + (m & 3)];
            const uint32_t S2 = vs[((2 + (m >> 2)) * 32 + lane) * 4 + (m & 3)];
            float sk;
            uint32_t b;
            if (!EDGE && !EXTM) {
                const float d = eval_interior(simple, false, S1, S2, rc.nw, rc.an, rc.gn, rc.bn2, pixel_f(P, m));
                b = __float_as_uint(d) >> 31;
                sk = fabsf(d) - T.bnd_c;
            } else {
                uint32_t n_m;
                float inv_m;
                count_of(lane, m, n_m, inv_m);
                b = eval_bounded<EXTM, uint32_t>(T, F, simple, n_m, inv_m, S1, S2, pixel_f(P, m), sk);
                if (EDGE && !(vmask >> m & 1u))
                    sk = 1.0f;  // columns past the row count as certified
            }
            if (sk > 0.0f)
                byte |= b << m;
            else
                und |= 1u << m;
        }
    }
    // the warp's list of uncertified (lane, pixel) pairs and their bits
    uint8_t *list = reinterpret_cast<uint8_t *>(slots + 384);
    uint8_t *res = list + 256;
    const uint32_t cnt = (uint32_t)__popc(und);
    const uint32_t incl = warp_incl_scan<uint32_t>(cnt, lane);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t at = incl - cnt;
    for (uint32_t u2 = und; u2; u2 &= u2 - 1)
        list[at++] = (uint8_t)(lane * 8 + (__ffs(u2) - 1));
    __syncwarp();
    Global G{};
    if constexpr (EXTM != 0)
        G = global_lms(*T.gs, T.N);
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
        const uint32_t e = r0 + lane < total ? list[r0 + lane] : (uint32_t)(lane * 8);
        const int own = (int)(e >> 3), m = (int)(e & 7u);
        const uint2 Pown = make_uint2(__shfl_sync(0xFFFFFFFFu, P.x, own), __shfl_sync(0xFFFFFFFFu, P.y, own));
        if (r0 + lane < total) {
            const uint32_t S1 = vs[((m >> 2) * 32 + own) * 4 + (m & 3)];
            const uint32_t S2 = vs[((2 + (m >> 2)) * 32 + own) * 4 + (m & 3)];
            uint32_t n_m;
            float inv_m;
            count_of(own, m, n_m, inv_m);
            if constexpr (EXTM != 0) {
                res[e] = (uint8_t)fp64_bit_ext(EXTM, (uint32_t)byte_at(Pown, m), S1, (uint64_t)S2, n_m, T.k, T.R,
                                               T.X.alpha1, T.X.k1, T.X.k2, T.X.gamma, T.X.p, T.X.q, G.L, G.M, G.S);
            } else {
                res[e] = (uint8_t)fp64_bit(T.method, (uint32_t)byte_at(Pown, m), S1, (uint64_t)S2, n_m, T.k, T.R);
            }
        }
    }
    __syncwarp();
    for (uint32_t u2 = und; u2; u2 &= u2 - 1) {
        const int m = __ffs(u2) - 1;
        byte |= (uint32_t)res[lane * 8 + m] << m;
    }
    __syncwarp();  // the list is rewritten by the next row
    return byte | (cnt << 8);
}

// Interior tiles, binarize modes, 32-bit S2: a one-row software pipeline.
// Iteration i computes the window sums of row i (slide, lane prefix, warp
// scan) and stores them to a warp-private shared-memory slot, then evaluates
// the threshold of row i-1 from the other slot.  The two halves are
// independent, and the loop body has no data-dependent branch except the
// rare FP64 near-tie path at its end, so the compiler can interleave the
// scan's latency chain with the threshold arithmetic.  Rows outside the image
// are handled without branches (safe row pointer + zero mask).
// EDGE: the same for the first and last tile columns (and tiles of images
// narrower than a tile): streams that leave the row are clamped and shifted
// (edge_clamp), the anchor window is clipped to the row, and the per-column
// counts and their reciprocals come from a per-warp table.
// smem: kPipeSlots x 16 = 11,520 bytes per warp (two 2 KB row slots, the 2 KB
// column table, 512 bytes for the FP64 near-tie list and its results, the
// 1 KB table of per-row constants and 3.75 KB for the parked loop state; the
// column-sum warm-up uses the first 4.5 KB before the row loop starts).
template <int MODE, bool WARMB = false, bool EDGE = false, int AW = 1, int EXTM = 0>
__device__ __forceinline__ void window_rows_pipe(const Image &g, const Window &win, const Thresh &T,
                                                 const Outputs &o, int64_t x0, int64_t y0,
                                                 int64_t y1, int lane, uint4 *slots,
                                                 const uint2 *stripe = nullptr)
{
    typedef uint32_t S2T;
    const int64_t H = g.H;
    const int64_t j0 = x0 + (int64_t)kColsPerLane * lane;
    const int l = win.l, r = win.r, oo = win.o, u = win.u;
    [[maybe_unused]] const size_t img_ext = dbg_image_extent(g);
    const int64_t colA = j0 + r, colB = j0 - l;
    // load columns (32-bit: the caller guarantees W <= 2^30) and, for EDGE,
    // the byte shifts of the A, B and centre streams as three signed bytes
    int32_t pA = (int32_t)colA, pB = (int32_t)colB, pP = (int32_t)j0;
    uint32_t shifts = 0;
    if (EDGE) {
        int64_t c;
        int sh;
        edge_clamp(colA, g.W, c, sh);
        pA = (int32_t)c;
        shifts = (uint32_t)(sh & 0xFF);
        edge_clamp(colB, g.W, c, sh);
        pB = (int32_t)c;
        shifts |= (uint32_t)(sh & 0xFF) << 8;
        edge_clamp(j0, g.W, c, sh);
        pP = (int32_t)c;
        shifts |= (uint32_t)(sh & 0xFF) << 16;
    }
    auto shift_of = [&](int q) { return (int)(int8_t)(uint8_t)(shifts >> (8 * q)); };
    const int kA = pA & 3, kB = pB & 3;  // warp-uniform unless EDGE
    const unsigned selA = (unsigned)kA * 0x1111u + 0x3210u;
    const unsigned selB = (unsigned)kB * 0x1111u + 0x3210u;
    auto ldA = [&](const uint8_t *rp) {
        const uint2 v = ld8_w3(rp + pA, kA, selA, g.img, img_ext);
        return EDGE ? shift8(v, shift_of(0)) : v;
    };
    auto ldB = [&](const uint8_t *rp) {
        const uint2 v = ld8_w3(rp + pB, kB, selB, g.img, img_ext);
        return EDGE ? shift8(v, shift_of(1)) : v;
    };

    // anchor words, read by the small-page warm-up only (the row loop takes
    // the anchor's bytes from the B streams, the column-sum warm-up from its
    // column sums): the caller guarantees (aend - a4) <= 128 AW, AW words per
    // lane (lane + 32 q); lanes past the window read the first word and mask
    // it to zero
    int64_t ac0 = x0 - l, aend = x0 + r;
    if (EDGE) {  // clip the anchor window to the row
        ac0 = ac0 > 0 ? ac0 : 0;
        aend = aend < g.W ? aend : g.W;
    }
    const int64_t a4 = ac0 & ~(int64_t)3;  // ac0 >= 0 here
    uint32_t keep[AW];
    int32_t aoff[AW];
#pragma unroll
    for (int q = 0; q < AW; q++) {
        const int64_t c4 = a4 + 4 * (lane + 32 * q);
        const bool has_word = c4 < aend;
        uint32_t kp = 0xFFFFFFFFu;
        if (c4 < ac0)
            kp &= 0xFFFFFFFFu << (8 * (int)(ac0 - c4));
        if (c4 + 4 > aend)
            kp = (c4 >= aend) ? 0u : (kp & (0xFFFFFFFFu >> (8 * (int)(c4 + 4 - aend))));
        keep[q] = kp;
        aoff[q] = (int32_t)(has_word ? c4 : a4);
    }
    auto anchor_row = [&](const uint8_t *rp, uint32_t &s1, uint32_t &s2) {
#pragma unroll
        for (int q = 0; q < AW; q++) {
            const uint32_t wd = (BZ_DBG_IN(rp + aoff[q], 4, g.img, img_ext, kDbgImage)
                                     ? __ldg(reinterpret_cast<const uint32_t *>(rp + aoff[q]))
                                     : 0u) &
                                keep[q];
            s1 = __dp4a(wd, 0x01010101u, s1);
            s2 = __dp4a(wd, wd, s2);
        }
    };

    // ---- warm-up (row y0), one row of look-ahead
    int32_t E1[kColsPerLane];
    uint32_t E2[kColsPerLane];
#pragma unroll
    for (int m = 0; m < kColsPerLane; m++) {
        E1[m] = 0;
        E2[m] = 0;
    }
    uint32_t a1p = 0, a2p = 0;
    if (stripe) {
        warm_from_stripes(stripe, g.W, colA, colB, ac0, aend, lane, E1, E2, a1p, a2p);
    } else {
        int64_t a_lo = y0 - oo + 1, a_hi = y0 + u;
        if (a_lo < 0)
            a_lo = 0;
        if (a_hi > H - 1)
            a_hi = H - 1;
        if (!WARMB) {
            warm_cols<AW, EDGE>(g, win, x0, lane, a_lo, a_hi, reinterpret_cast<uint32_t *>(slots), E1, E2, a1p,
                                a2p);
        } else {  // small pages: eight rows per batch of loads (latency-bound tiles of 1-4 rows)
            const uint2 Z = make_uint2(0u, 0u);
            for (int64_t a = a_lo; a <= a_hi; a += kWarmRows) {
                uint2 Ar[kWarmRows], Br[kWarmRows];
                uint32_t w1r[kWarmRows], w2r[kWarmRows];
#pragma unroll
                for (int q = 0; q < kWarmRows; q++) {
                    Ar[q] = Br[q] = Z;
                    w1r[q] = w2r[q] = 0u;
                    if (a + q <= a_hi) {  // warp-uniform
                        const uint8_t *rp = g.img + (a + q) * g.pitch;
                        Ar[q] = ldA(rp);
                        Br[q] = ldB(rp);
                        anchor_row(rp, w1r[q], w2r[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < kWarmRows; q += 4) {  // rows past a_hi are zero
                    const uint2 A4[4] = {Ar[q], Ar[q + 1], Ar[q + 2], Ar[q + 3]};
                    const uint2 B4[4] = {Br[q], Br[q + 1], Br[q + 2], Br[q + 3]};
                    warm8x4(A4, B4, E1, E2);
                }
#pragma unroll
                for (int q = 0; q < kWarmRows; q++) {
                    a1p += w1r[q];
                    a2p += w2r[q];
                }
            }
        }
    }
    uint32_t A1 = __reduce_add_sync(0xFFFFFFFFu, a1p);
    S2T A2 = (S2T)__reduce_add_sync(0xFFFFFFFFu, a2p);  // < 2^32 when h*w <= 66051

    // The anchor's entering and leaving bytes are already in the B streams:
    // byte m of lane L's B stream is column x0 + 8 L + m - l, which lies in
    // the anchor window [x0 - l, x0 + r) exactly when 8 L + m < w (w <= 256
    // on this path; edge tiles read columns outside [0, W) as 0, as the
    // clipped anchor window does).  amx / amy: those bytes of the lane.
    const int anb = win.w - kColsPerLane * lane;
    const uint32_t amx = anb >= 4 ? 0xFFFFFFFFu : (anb <= 0 ? 0u : 0xFFFFFFFFu >> (8 * (4 - anb)));
    const uint32_t amy = anb >= 8 ? 0xFFFFFFFFu : (anb <= 4 ? 0u : 0xFFFFFFFFu >> (8 * (8 - anb)));

    // branch-free slide data for row i: rows outside the image read row 0
    // and are masked to zero
    uint2 nA, nB, nC, nD;
    uint32_t nd1, nd2;
    auto fetch = [&](int64_t i) {
        const int64_t ra = i + u, rb = i - oo;
        const bool va = ra < H, vb = rb >= 0;
        const uint8_t *pa = g.img + (va ? ra : 0) * g.pitch;
        const uint8_t *pb = g.img + (vb ? rb : 0) * g.pitch;
        uint2 A = ldA(pa), B = ldB(pa);
        uint2 C = ldA(pb), D = ldB(pb);
        const uint32_t ma = va ? 0xFFFFFFFFu : 0u, mb = vb ? 0xFFFFFFFFu : 0u;
        nA = make_uint2(A.x & ma, A.y & ma);
        nB = make_uint2(B.x & ma, B.y & ma);
        nC = make_uint2(C.x & mb, C.y & mb);
        nD = make_uint2(D.x & mb, D.y & mb);
        // the anchor's row change: its bytes of the entering row minus those
        // of the leaving row
        const uint32_t bx = nB.x & amx, by = nB.y & amy, dx = nD.x & amx, dy = nD.y & amy;
        nd1 = __dp4a(bx, 0x01010101u, __dp4a(by, 0x01010101u, 0u)) -
              __dp4a(dx, 0x01010101u, __dp4a(dy, 0x01010101u, 0u));
        nd2 = __dp4a(bx, bx, __dp4a(by, by, 0u)) - __dp4a(dx, dx, __dp4a(dy, dy, 0u));
    };

    // window sums of the current row -> slot (i & 1)
    auto sums_to_slot = [&](int64_t i) {
        uint32_t p1[kColsPerLane], p2[kColsPerLane];
        uint32_t run1 = 0, run2 = 0;
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            run1 += (uint32_t)E1[m];
            run2 += E2[m];
            p1[m] = run1;
            p2[m] = run2;
        }
        const uint32_t inc1 = warp_incl_scan<uint32_t>(run1, lane);
        const uint32_t inc2 = warp_incl_scan<uint32_t>(run2, lane);
        const uint32_t off1 = A1 + (inc1 - run1);
        const uint32_t off2 = A2 + (inc2 - run2);
        uint4 *sl = slots + (int)(i & 1) * 128;
        sl[0 * 32 + lane] = make_uint4(off1 + p1[0], off1 + p1[1], off1 + p1[2], off1 + p1[3]);
        sl[1 * 32 + lane] = make_uint4(off1 + p1[4], off1 + p1[5], off1 + p1[6], off1 + p1[7]);
        sl[2 * 32 + lane] = make_uint4(off2 + p2[0], off2 + p2[1], off2 + p2[2], off2 + p2[3]);
        sl[3 * 32 + lane] = make_uint4(off2 + p2[4], off2 + p2[5], off2 + p2[6], off2 + p2[7]);
    };

    const bool simple = !EXTM && T.method == 0 && T.alpha >= 0.0f && T.beta >= 0.0f;
    // EXTM: a Table 1 method other than Sauvola / Niblack (T is then a
    // ThreshExt): its FP32 constants from the global statistics
    const ThreshExt &TX = static_cast<const ThreshExt &>(T);
    ExtF F{};
    if (EXTM)
        F = make_extf(EXTM, T.k, T.R, TX.X, global_lms(*TX.gs, TX.N), T.eps);
    unsigned long long nfb = 0;

    // EDGE: column counts of this lane's 8 columns (1 past the row) and
    // their correctly rounded reciprocals, entry m * 32 + lane; each lane
    // reads back only its own entries.  `vmask`: the output bits inside the
    // row.
    uint2 *ctab = reinterpret_cast<uint2 *>(slots + 256);
    uint32_t vmask = 0xFFu;
    if (EDGE) {
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            const int64_t j = j0 + m;
            const int64_t c = (j + r < g.W - 1 ? j + r : g.W - 1) - (j - l > -1 ? j - l : -1);
            const uint32_t cm = j < g.W ? (uint32_t)c : 1u;
            ctab[m * 32 + lane] = make_uint2(__float_as_uint(__frcp_rn((float)cm)), cm);
        }
        const int64_t left = g.W - j0;
        vmask = left >= 8 ? 0xFFu : (left <= 0 ? 0u : (1u << (unsigned)left) - 1u);
    }

    // The per-row constants of the threshold, 32 rows at a time (one row per
    // lane) in the warp's shared memory, read back with two broadcast loads
    // per row: the clipped row count, n = rows * w, 1/n from correctly rounded
    // reciprocals (EDGE: 1/rows, the column factor comes from the table), the
    // interior form's alpha/n, gamma/n and beta/n^2, and the output row's
    // offset.  Computed in each row instead, they cost every lane ~40
    // instructions per row (64-bit clipping, the reciprocal's fix-up).
    RowC *rtab = reinterpret_cast<RowC *>(slots + kPipeSlotsRows);
    auto fill_rows = [&](int64_t i0) {
        __syncwarp();  // the previous 32 rows' entries are read
        const int64_t i = i0 + lane;
        if (i < y1) {
            const float inv_w = __frcp_rn((float)win.w);
            const float inv_h = __frcp_rn((float)win.h);
            const int64_t rows = (i + u < H - 1 ? i + u : H - 1) - (i - oo > -1 ? i - oo : -1);
            RowC c;
            c.nrow = (uint32_t)rows;
            c.nw = c.nrow * (uint32_t)win.w;
            c.inv_nw = c.nrow == (uint32_t)win.h ? (EDGE ? inv_h : inv_h * inv_w)
                                                 : __frcp_rn((float)rows) * (EDGE ? 1.0f : inv_w);
            c.an = T.alpha * c.inv_nw;
            c.gn = T.gamma * c.inv_nw;
            c.bn2 = (T.beta * c.inv_nw) * c.inv_nw;
            c.dst = (i - o.out_row0) * o.out_pitch;
            rtab[lane] = c;
        }
        __syncwarp();
    };

    // FP32 threshold of row i from slot (i & 1) and its pixels P.  Stores the
    // byte and returns false when every pixel of the warp's row is certified
    // (always outside MODE_FP64); else returns true with the FP32 byte and
    // the lane's smallest slack in byte_out / slack_out, stored by
    // threshold_rare after the near-tie path.
    auto threshold_fast = [&](int64_t i, uint2 P, uint32_t &byte_out, float &slack_out) -> bool {
        if ((((int)(i - y0)) & 31) == 0)  // warp-uniform
            fill_rows(i);
        const uint4 *sl = slots + (int)(i & 1) * 128;
        const uint4 s1a = sl[0 * 32 + lane], s1b = sl[1 * 32 + lane];
        const uint4 s2a = sl[2 * 32 + lane], s2b = sl[3 * 32 + lane];
        const uint32_t S1v[8] = {s1a.x, s1a.y, s1a.z, s1a.w, s1b.x, s1b.y, s1b.z, s1b.w};
        const uint32_t S2v[8] = {s2a.x, s2a.y, s2a.z, s2a.w, s2b.x, s2b.y, s2b.z, s2b.w};
        const RowC rc = rtab[((int)(i - y0)) & 31];
        const uint32_t nrow = rc.nrow;
        const uint32_t nw = rc.nw;
        const float inv_nw = rc.inv_nw;
        // count and 1/count of column m: the window width (interior tiles) or
        // the table entry (edge tiles)
        auto count_of = [&](int ln, int m, uint32_t &n_m, float &inv_m) {
            if (EDGE) {
                const uint2 e = ctab[m * 32 + ln];
                n_m = nrow * e.y;
                inv_m = inv_nw * __uint_as_float(e.x);
            } else {
                n_m = nw;
                inv_m = inv_nw;
            }
        };
        auto count = [&](int m, uint32_t &n_m, float &inv_m) { count_of(lane, m, n_m, inv_m); };
        // interior tiles: t / n per unit of S1 from row constants, so that a
        // pixel costs d = t - I = S1 (alpha/n + beta/n^2 sqrt(V)) - I (Sauvola
        // with alpha, beta >= 0), else alpha S1/n + (beta S1/n^2 + gamma/n)
        // sqrt(V) - I; certified when |d| > T.bnd_c
        const float an = rc.an, gn = rc.gn, bn2 = rc.bn2;
        // V = n S2 - S1^2 < n^2 255^2 / 4: below 2^32 when n <= 513, so
        // that wrapping 32-bit products give it exactly (V32)
        auto eval_n = [&](bool SIMPLE, bool V32, int m, uint32_t S1, uint32_t S2) -> float {
            return eval_interior(SIMPLE, V32, S1, S2, nw, an, gn, bn2, pixel_f(P, m));
        };
        // FP32 threshold of pixel m: returns its bit and sets `slack` =
        // |d| - E, certified when > 0 (columns past the row count as
        // certified).  SIMPLE: Sauvola with alpha, beta >= 0 (mag = t).
        auto eval = [&](bool SIMPLE, int m, uint32_t S1, uint32_t S2, float &slack) -> uint32_t {
            uint32_t n_m;
            float inv_m;
            count(m, n_m, inv_m);
            const uint32_t b = eval_bounded<EXTM, S2T>(T, F, SIMPLE, n_m, inv_m, S1, S2, pixel_f(P, m), slack);
            if (EDGE && !(vmask >> m & 1u))
                slack = 1.0f;
            return b;
        };
        // hot path: the bits and the row's smallest slack only
        uint32_t byte = 0;
        float minslack = 1.0f;
        if (!EDGE && !EXTM) {
            float mind = 3.0e38f;  // the row's smallest |d| (one min per pixel)
            auto row8 = [&](bool SIMPLE, bool V32) {
#pragma unroll
                for (int m = kColsPerLane - 1; m >= 0; m--) {
                    const float d = eval_n(SIMPLE, V32, m, S1v[m], S2v[m]);
                    byte = (byte << 1) | (__float_as_uint(d) >> 31);
                    mind = fminf(mind, fabsf(d));
                }
            };
            const bool v32 = nw <= 513u;
            if (simple) {
                if (v32)
                    row8(true, true);
                else
                    row8(true, false);
            } else {
                if (v32)
                    row8(false, true);
                else
                    row8(false, false);
            }
            minslack = mind <= T.bnd_c ? -1.0f : 1.0f;
        } else if (simple) {
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                float sk;
                byte |= eval(true, m, S1v[m], S2v[m], sk) << m;
                minslack = fminf(minslack, sk);
            }
        } else {
#pragma unroll
            for (int m = 0; m < kColsPerLane; m++) {
                float sk;
                byte |= eval(false, m, S1v[m], S2v[m], sk) << m;
                minslack = fminf(minslack, sk);
            }
        }
        if (MODE == MODE_FP64 && __any_sync(0xFFFFFFFFu, !(minslack > 0.0f))) {
            byte_out = byte;
            slack_out = minslack;
            return true;
        }
        uint8_t *dst = o.bits + rc.dst + ((j0 >> 3) - o.out_byte0);
        if ((!EDGE || vmask) && BZ_DBG_IN(dst, 1, o.bits, o.bits_bytes, kDbgOutput))
            *dst = (uint8_t)(EDGE ? (byte & vmask) : byte);
        return false;
    };
    // the near-tie path of row i (the whole warp), then the byte's store
    auto threshold_rare = [&](int64_t i, uint2 P, uint32_t byte, float minslack) {
        const RowC rc = rtab[((int)(i - y0)) & 31];
        uint32_t rb;
        if constexpr (EXTM != 0)
            rb = near_tie_row<EDGE, EXTM, ThreshExt>(TX, F, slots, (int)(i & 1), lane, P, byte, !(minslack > 0.0f),
                                                     rc, simple, vmask);
        else
            rb = near_tie_row<EDGE, 0, Thresh>(T, F, slots, (int)(i & 1), lane, P, byte, !(minslack > 0.0f), rc,
                                               simple, vmask);
        byte = rb & 0xFFu;
        nfb += rb >> 8;
        uint8_t *dst = o.bits + rc.dst + ((j0 >> 3) - o.out_byte0);
        if ((!EDGE || vmask) && BZ_DBG_IN(dst, 1, o.bits, o.bits_bytes, kDbgOutput))
            *dst = (uint8_t)(EDGE ? (byte & vmask) : byte);
    };

    auto centre = [&](int64_t i) {
        if (EDGE)
            return shift8(ld8_w3(g.img + i * g.pitch + pP, pP & 3, (unsigned)(pP & 3) * 0x1111u + 0x3210u,
                                 g.img, img_ext),
                          shift_of(2));
        if (!BZ_DBG_IN(g.img + i * g.pitch + j0, 8, g.img, img_ext, kDbgImage))
            return make_uint2(0u, 0u);
        return __ldg(reinterpret_cast<const uint2 *>(g.img + i * g.pitch + j0));
    };

    // The loop state parks in the warp's shared memory while a near-tie row
    // is decided (word w of the lane at w * 32 + lane), so that the near-tie
    // path finds the registers free and the row loop's allocation does not
    // have to keep its state alive across that path (which, kept live across
    // it, cost the loop ~3 % of its time with no near-tie taken).
    volatile uint32_t *park = reinterpret_cast<volatile uint32_t *>(slots + kPipeSlotsPark);
    uint2 Pprev = make_uint2(0u, 0u);  // row y0's pixels, set by the prologue below
    auto park_state = [&]() {
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            park[m * 32 + lane] = (uint32_t)E1[m];
            park[(8 + m) * 32 + lane] = E2[m];
        }
        const uint32_t w[14] = {A1, (uint32_t)A2, nA.x, nA.y, nB.x, nB.y, nC.x, nC.y, nD.x, nD.y, nd1, nd2,
                                Pprev.x, Pprev.y};
#pragma unroll
        for (int k = 0; k < 14; k++)
            park[(16 + k) * 32 + lane] = w[k];
    };
    auto unpark_state = [&]() {
#pragma unroll
        for (int m = 0; m < kColsPerLane; m++) {
            E1[m] = (int32_t)park[m * 32 + lane];
            E2[m] = park[(8 + m) * 32 + lane];
        }
        uint32_t w[14];
#pragma unroll
        for (int k = 0; k < 14; k++)
            w[k] = park[(16 + k) * 32 + lane];
        A1 = w[0];
        A2 = (S2T)w[1];
        nA = make_uint2(w[2], w[3]);
        nB = make_uint2(w[4], w[5]);
        nC = make_uint2(w[6], w[7]);
        nD = make_uint2(w[8], w[9]);
        nd1 = w[10];
        nd2 = w[11];
        Pprev = make_uint2(w[12], w[13]);
    };

    // prologue: row y0
    sums_to_slot(y0);
    Pprev = centre(y0);
    if (y0 + 1 < y1)
        fetch(y0 + 1);
    int64_t i = y0 + 1;
    for (;;) {
        // rows until one with a near-tie (warp-uniform exit)
        bool tie = false;
        uint2 Ptie = make_uint2(0u, 0u);
        uint32_t tbyte = 0;
        float tslack = 1.0f;
        for (; i < y1; i++) {
            const uint2 Pcur = centre(i);
            slide8(nA, nB, nC, nD, E1, E2);
            A1 += (uint32_t)__reduce_add_sync(0xFFFFFFFFu, nd1);
            A2 += (S2T)__reduce_add_sync(0xFFFFFFFFu, nd2);
            fetch(i + 1 < y1 ? i + 1 : i);  // the last fetch is unused (no branch)
            sums_to_slot(i);
            const uint2 Prow = Pprev;
            Pprev = Pcur;
            if (threshold_fast(i - 1, Prow, tbyte, tslack)) {
                Ptie = Prow;
                tie = true;
                break;
            }
        }
        if (MODE != MODE_FP64 || !tie)
            break;
        park_state();
        threshold_rare(i - 1, Ptie, tbyte, tslack);
        unpark_state();
        i++;
    }
    {
        uint32_t tbyte;
        float tslack;
        if (threshold_fast(y1 - 1, Pprev, tbyte, tslack))
            threshold_rare(y1 - 1, Pprev, tbyte, tslack);
    }

    if (MODE == MODE_FP64 && o.fallbacks) {
        const unsigned v = __reduce_add_sync(0xFFFFFFFFu, (unsigned)nfb);
        if (lane == 0 && v)
            atomicAdd(o.fallbacks, (unsigned long long)v);
    }
}

// The tiles of one launch.  Edge tiles (the first and last tile columns)
// clamp their byte streams and look up per-column counts, or take the
// generic path, so they take longer per row; with a one-wave grid the
// slowest warps set the launch's duration.  A balanced schedule therefore
// gives the two edge columns shorter tiles (edge_h < tile_h rows) and lists
// them first (n_edge tiles, alternating left and right column); the uniform
// schedule has n_edge = 0 and every column in the tile_h grid.
struct TileSched {
    int64_t tiles_x, tile_h, edge_h, n_edge, tiles_total, row0, row1;
    int64_t tx0;   // first tile column (column-band launches; else 0)
    int prefetch;  // tiles start with an L2 prefetch of their input
};

// Tile t of a schedule: column tx, rows [y0, y1), and its stripe sums st
// (uniform schedules with a stripe pre-pass only; else nullptr).
__device__ __forceinline__ void sched_tile(const TileSched &S, int64_t W, const uint2 *stripes, int64_t t,
                                           int64_t &tx, int64_t &y0, int64_t &y1, const uint2 *&st)
{
    st = nullptr;
    if (t < S.n_edge) {
        tx = (t & 1) ? S.tiles_x - 1 : 0;
        y0 = S.row0 + (t >> 1) * S.edge_h;
        y1 = y0 + S.edge_h;
    } else {
        const int64_t t2 = t - S.n_edge;
        const int64_t ncol = S.n_edge ? S.tiles_x - 2 : S.tiles_x;
        const int64_t ty = t2 / ncol;
        tx = (S.n_edge ? 1 : 0) + (t2 - ty * ncol);
        y0 = S.row0 + ty * S.tile_h;
        y1 = y0 + S.tile_h;
        if (stripes)
            st = stripes + ty * W;
    }
    tx += S.tx0;
    if (y1 > S.row1)
        y1 = S.row1;
}

// Whether the pipelined path applies to a launch (host and device): binarize
// modes, 32-bit S2, aligned 8-byte loads, W in [8, 2^30], and an anchor
// window [x0 - l, x0 + r) that AW words per lane cover: at most 128 AW bytes
// from the word boundary below x0 - l (x0 is a multiple of 256; an edge
// tile's clipped window starts at column 0 or there, and it is no wider).
// AW also sets the halo of the column-sum warm-up (64 AW columns each side,
// l, r <= 64 AW).  Returns AW (1 or 2), or 0 when the path does not apply.
__host__ __device__ inline int pipe_words(int mode, bool vec, bool s2_32, const Image &g,
                                          const Window &win)
{
    if (!((mode == MODE_FP64 || mode == MODE_FP32) && vec && s2_32 && g.W >= 8 &&
          g.W <= ((int64_t)1 << 30) && win.l <= kTileCols))
        return 0;
    const int span = win.w + ((4 - (win.l & 3)) & 3);
    return span <= 128 ? 1 : (span <= 256 ? 2 : 0);
}

// Ask L2 for every input byte a tile will read (rows y0 - o + 1 .. y1 - 1 + u,
// columns x0 - l .. x0 + 255 + r, clipped to the image), one bulk prefetch
// per row, so that the warm-up and slide loads of a launch whose image is not
// in L2 yet wait for L2 rather than for HBM.  Each prefetched range is the
// row's span rounded out to 16-byte blocks, which stay inside the blocks
// that hold its first and last bytes.
__device__ __forceinline__ void tile_prefetch_l2(const Image &g, const Window &win, int64_t x0, int64_t y0,
                                                 int64_t y1, int lane)
{
    int64_t r0 = y0 - win.o + 1, r1 = y1 - 1 + win.u;  // inclusive
    r0 = r0 < 0 ? 0 : r0;
    r1 = r1 > g.H - 1 ? g.H - 1 : r1;
    int64_t c0 = x0 - win.l, c1 = x0 + kTileCols + win.r;  // [c0, c1)
    c0 = c0 < 0 ? 0 : c0;
    c1 = c1 > g.W ? g.W : c1;
    if (c0 >= c1)
        return;
    for (int64_t row = r0 + lane; row <= r1; row += 32) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(g.img + row * g.pitch + c0) & ~(uintptr_t)15;
        const uintptr_t e = (reinterpret_cast<uintptr_t>(g.img + row * g.pitch + c1) + 15) & ~(uintptr_t)15;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
    }
}

// One warp computes the tile of columns [x0, x0+256) x rows [y0, y1).
// prefetch: start with tile_prefetch_l2.
// AW > 0: the launch takes the pipelined path with AW anchor words per lane
// (pipe_words: the anchor and halo width) and the caller provides
// kPipeSlots x 16 bytes of shared memory per warp (`slots`); interior and
// edge tiles then both take it.  AW = 0: window_rows.
template <int MODE, bool VEC, typename S2T, int AW, bool WARMB = false>
__device__ __forceinline__ void window_tile(const Image &g, const Window &win, const Thresh &T,
                                            const Outputs &o, int64_t x0, int64_t y0, int64_t y1,
                                            int lane, uint4 *slots, const uint2 *stripe = nullptr,
                                            bool prefetch = false)
{
    if (prefetch)
        tile_prefetch_l2(g, win, x0, y0, y1, lane);
    // interior: left edge stream of lane 0 and right edge stream of lane 31
    // inside the row, and the whole tile left of the last column
    const bool interior = VEC && (x0 - win.l >= 0) && (x0 + kTileCols + win.r <= g.W);
    if (AW > 0) {
        constexpr int kAW = AW > 0 ? AW : 1;
        if (interior)
            window_rows_pipe<MODE, WARMB, false, kAW>(g, win, T, o, x0, y0, y1, lane, slots, stripe);
        else
            window_rows_pipe<MODE, WARMB, true, kAW>(g, win, T, o, x0, y0, y1, lane, slots, stripe);
    } else if (interior) {
        window_rows<MODE, VEC, true, S2T, false, WARMB>(g, win, T, o, x0, y0, y1, lane, stripe);
    } else {
        window_rows<MODE, VEC, false, S2T, false, WARMB>(g, win, T, o, x0, y0, y1, lane, stripe);
    }
}

}  // namespace bz
