/*
 * Oracle for local adaptive binarization (Chan, "Memory-efficient and fast
 * implementation of local adaptive binarization methods", arXiv 1905.13038).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU library computes.  Only the test-suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or helper with the CUDA library and must
 * never be linked into it.
 *
 * Build: plain C11, -O2 -ffp-contract=off (no FMA contraction, no fast-math)
 * so that every double operation is one IEEE-754 binary64 operation rounded to
 * nearest-even, on x86-64 and on aarch64 alike.
 *
 * Conventions (shared with the paper):
 *   image I: H rows x W columns of 8-bit gray levels, row pitch >= W bytes.
 *   window h x w (h rows, w columns); Algorithm 1 parameters
 *     l = floor((w+1)/2), r = floor(w/2), o = floor((h+1)/2), u = floor(h/2);
 *   the window of pixel (i,j) is rows (i-o, i+u] x columns (j-l, j+r]
 *     (Sec. 1 definition of m and s; Sec. 3.1 identities).
 *   Border rule: pixels outside the image are 0 (Sec. 3.2 assumptions) and
 *     the count n is the number of in-image window pixels (Algorithm 1).
 *   S1 = sum I, S2 = sum I^2, n, V = n*S2 - S1^2 (= n^2 * variance).
 *   Output bit = 0 where I <= t (dark, "foreground"), 1 elsewhere (Algorithm 1).
 *   Packed output: bit (j & 7) of byte (j >> 3) of the row, LSB first,
 *     padding bits 0.
 *
 * The paper does not fix a floating-point evaluation order for the
 * threshold; this file evaluates it in IEEE binary64, round to nearest, every
 * operation rounded and none contracted, in this order:
 *     nd = n; m = S1/nd; s = sqrt(V/(nd*nd));
 *     Sauvola t = m*(1 + k*(s/R - 1));   Niblack t = m + k*s.
 * In exact arithmetic this equals the Sec. 1 definition since s^2 = S2/n - m^2.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Window parameters: Algorithm 1, first four assignments.                    */
/* ------------------------------------------------------------------------ */
void oracle_window_params(int32_t h, int32_t w, int32_t *l, int32_t *r,
                          int32_t *o, int32_t *u)
{
    *l = (w + 1) / 2;
    *r = w / 2;
    *o = (h + 1) / 2;
    *u = h / 2;
}

/* Gray level with the "undefined elements are zero" rule (Sec. 3.2). */
static inline uint32_t px(const uint8_t *img, int64_t H, int64_t W,
                          int64_t pitch, int64_t i, int64_t j)
{
    if (i < 0 || i >= H || j < 0 || j >= W)
        return 0;
    return img[i * pitch + j];
}

static int check_args(int64_t H, int64_t W, int64_t pitch, int32_t h, int32_t w)
{
    if (H < 1 || W < 1 || pitch < W || h < 1 || w < 1)
        return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (i) Definitive implementation: direct summation over the clipped window   */
/*     (Sec. 1 formulas for m and s; Theta(HWhw) time).                      */
/* ------------------------------------------------------------------------ */
int oracle_window_sums_bruteforce(const uint8_t *img, int64_t H, int64_t W,
                                  int64_t pitch, int32_t h, int32_t w,
                                  uint32_t *S1, uint64_t *S2, uint32_t *n)
{
    if (check_args(H, W, pitch, h, w))
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            uint64_t s1 = 0, s2 = 0, cnt = 0;
            for (int64_t a = i - o + 1; a <= i + u; a++) {
                for (int64_t b = j - l + 1; b <= j + r; b++) {
                    if (a < 0 || a >= H || b < 0 || b >= W)
                        continue;
                    uint64_t v = img[a * pitch + b];
                    s1 += v;
                    s2 += v * v;
                    cnt += 1;
                }
            }
            S1[i * W + j] = (uint32_t)s1;
            S2[i * W + j] = s2;
            n[i * W + j] = (uint32_t)cnt;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (ii) Integral images (Sec. 2): J_{i,j} = sum_{a<=i, b<=j} f(I_{a,b}) with  */
/*      J = 0 for negative indices, built by the Sec. 2 recurrence; a window */
/*      sum is the four-corner difference.  int64 as Sec. 3.3 requires.      */
/* ------------------------------------------------------------------------ */
static int64_t J_at(const int64_t *J, int64_t H, int64_t W, int64_t i, int64_t j)
{
    if (i < 0 || j < 0)
        return 0;
    if (i >= H)
        i = H - 1; /* beyond the last row the image is zero: J stops growing */
    if (j >= W)
        j = W - 1;
    return J[i * W + j];
}

int oracle_window_sums_integral(const uint8_t *img, int64_t H, int64_t W,
                                int64_t pitch, int32_t h, int32_t w,
                                uint32_t *S1, uint64_t *S2, uint32_t *n)
{
    if (check_args(H, W, pitch, h, w))
        return 1;
    int64_t *J1 = (int64_t *)malloc((size_t)(H * W) * sizeof(int64_t));
    int64_t *J2 = (int64_t *)malloc((size_t)(H * W) * sizeof(int64_t));
    if (!J1 || !J2) {
        free(J1);
        free(J2);
        return 2;
    }
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            int64_t f1 = img[i * pitch + j];
            int64_t f2 = f1 * f1;
            int64_t up1 = i > 0 ? J1[(i - 1) * W + j] : 0;
            int64_t lf1 = j > 0 ? J1[i * W + j - 1] : 0;
            int64_t ul1 = (i > 0 && j > 0) ? J1[(i - 1) * W + j - 1] : 0;
            int64_t up2 = i > 0 ? J2[(i - 1) * W + j] : 0;
            int64_t lf2 = j > 0 ? J2[i * W + j - 1] : 0;
            int64_t ul2 = (i > 0 && j > 0) ? J2[(i - 1) * W + j - 1] : 0;
            J1[i * W + j] = up1 + lf1 + f1 - ul1;
            J2[i * W + j] = up2 + lf2 + f2 - ul2;
        }
    }
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            int64_t a0 = i - o, a1 = i + u, b0 = j - l, b1 = j + r;
            int64_t s1 = J_at(J1, H, W, a1, b1) - J_at(J1, H, W, a0, b1) -
                         J_at(J1, H, W, a1, b0) + J_at(J1, H, W, a0, b0);
            int64_t s2 = J_at(J2, H, W, a1, b1) - J_at(J2, H, W, a0, b1) -
                         J_at(J2, H, W, a1, b0) + J_at(J2, H, W, a0, b0);
            /* the count is the same four-corner difference with f = 1 on the
               image, i.e. the clipped rectangle area */
            int64_t ra = (a1 < H - 1 ? a1 : H - 1) - (a0 > -1 ? a0 : -1);
            int64_t cb = (b1 < W - 1 ? b1 : W - 1) - (b0 > -1 ? b0 : -1);
            S1[i * W + j] = (uint32_t)s1;
            S2[i * W + j] = (uint64_t)s2;
            n[i * W + j] = (uint32_t)(ra * cb);
        }
    }
    free(J1);
    free(J2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (iii) The paper's recursive scheme (Sec. 3.1 identities, Algorithm 1).    */
/*                                                                           */
/* Stripe level: for every column j keep C_j = sum of I over rows            */
/*   (i-o, i+u] and D_j the same sum of I^2; moving from row i-1 to row i     */
/*   adds row i+u and removes row i-o.                                       */
/* Window level: along a row keep c = sum of C_b over columns (j-l, j+r] and */
/*   d the same over D_b; moving from column j-1 to j adds column j+r and    */
/*   removes column j-l.                                                     */
/* Before the first row, C_j holds rows [0, u) so that the first update      */
/* (adding row u, removing row -o = 0) yields rows (-o, u]; before the first */
/* column, c holds columns [0, r) for the same reason.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t H, W, pitch;
    int32_t l, r, o, u;
    const uint8_t *img;
    uint32_t *C; /* stripe sums of I,   length W */
    uint32_t *D; /* stripe sums of I^2, length W */
} stripe_state;

/* Columns sums for rows [first_row, first_row + count): warm-up used before
 * a row band starts at first_row + count == band start + u. */
static void stripe_init(stripe_state *st, int64_t first_row, int64_t count)
{
    for (int64_t j = 0; j < st->W; j++) {
        uint32_t Cj = 0, Dj = 0;
        for (int64_t a = first_row; a < first_row + count; a++) {
            uint32_t v = px(st->img, st->H, st->W, st->pitch, a, j);
            Cj += v;
            Dj += v * v;
        }
        st->C[j] = Cj;
        st->D[j] = Dj;
    }
}

/* Stripe level, second identity of Sec. 3.1: slide every column sum down to
 * the window rows of image row i. */
static void stripe_advance(stripe_state *st, int64_t i)
{
    for (int64_t j = 0; j < st->W; j++) {
        uint32_t add = px(st->img, st->H, st->W, st->pitch, i + st->u, j);
        uint32_t sub = px(st->img, st->H, st->W, st->pitch, i - st->o, j);
        st->C[j] = st->C[j] + add - sub;
        st->D[j] = st->D[j] + add * add - sub * sub;
    }
}

static inline uint32_t Cat(const stripe_state *st, int64_t j)
{
    return (j < 0 || j >= st->W) ? 0 : st->C[j];
}
static inline uint32_t Dat(const stripe_state *st, int64_t j)
{
    return (j < 0 || j >= st->W) ? 0 : st->D[j];
}

/* Clipped count n of Algorithm 1. */
static inline uint32_t count_n(int64_t i, int64_t j, int64_t H, int64_t W,
                               int32_t l, int32_t r, int32_t o, int32_t u)
{
    int64_t cols = (j + r < W - 1 ? j + r : W - 1) - (j - l > -1 ? j - l : -1);
    int64_t rows = (i + u < H - 1 ? i + u : H - 1) - (i - o > -1 ? i - o : -1);
    return (uint32_t)(cols * rows);
}

/* Window level for one row: the first identity of Sec. 3.1, emitting
 * (S1, S2, n) for each column through the callback arrays. */
static void window_row(const stripe_state *st, int64_t i, uint32_t *S1row,
                       uint64_t *S2row, uint32_t *nrow)
{
    uint32_t c = 0;
    uint64_t d = 0;
    for (int64_t b = 0; b < st->r; b++) {
        c += Cat(st, b);
        d += Dat(st, b);
    }
    for (int64_t j = 0; j < st->W; j++) {
        c = c + Cat(st, j + st->r) - Cat(st, j - st->l);
        d = d + Dat(st, j + st->r) - Dat(st, j - st->l);
        S1row[j] = c;
        S2row[j] = d;
        nrow[j] = count_n(i, j, st->H, st->W, st->l, st->r, st->o, st->u);
    }
}

int oracle_window_sums_recursive(const uint8_t *img, int64_t H, int64_t W,
                                 int64_t pitch, int32_t h, int32_t w,
                                 uint32_t *S1, uint64_t *S2, uint32_t *n)
{
    if (check_args(H, W, pitch, h, w))
        return 1;
    stripe_state st;
    st.H = H;
    st.W = W;
    st.pitch = pitch;
    st.img = img;
    oracle_window_params(h, w, &st.l, &st.r, &st.o, &st.u);
    st.C = (uint32_t *)malloc((size_t)W * sizeof(uint32_t));
    st.D = (uint32_t *)malloc((size_t)W * sizeof(uint32_t));
    if (!st.C || !st.D) {
        free(st.C);
        free(st.D);
        return 2;
    }
    stripe_init(&st, 0, st.u);
    for (int64_t i = 0; i < H; i++) {
        stripe_advance(&st, i);
        window_row(&st, i, S1 + i * W, S2 + i * W, n + i * W);
    }
    free(st.C);
    free(st.D);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (v) Canonical FP64 thresholds (Sec. 1 Sauvola formula; Table 1 Niblack).  */
/* ------------------------------------------------------------------------ */
static inline int64_t variance_numerator(uint32_t S1, uint64_t S2, uint32_t n)
{
    return (int64_t)n * (int64_t)S2 - (int64_t)S1 * (int64_t)S1;
}

double oracle_threshold(int32_t method, uint32_t S1, uint64_t S2, uint32_t n,
                        double k, double R)
{
    int64_t V = variance_numerator(S1, S2, n);
    double nd = (double)n;
    double m = (double)S1 / nd;
    double s = sqrt((double)V / (nd * nd));
    if (method == ORACLE_SAUVOLA)
        return m * (1.0 + k * (s / R - 1.0));
    return m + k * s; /* Niblack */
}

static inline uint8_t decide(uint32_t I, double t)
{
    return ((double)I <= t) ? 0 : 1;
}

/* The paper's own floating-point order in Algorithm 1: m = c/n,
 * v = d/n - m^2, and the square-root-free Sauvola condition of Sec. 3.2.
 * Reported for comparison only; it may differ from the canonical order by
 * rounding (v can cancel catastrophically). */
uint8_t oracle_sauvola_bit_paper_order(uint32_t I, uint32_t S1, uint64_t S2,
                                       uint32_t n, double k, double R)
{
    double c = (double)S1, d = (double)S2, nd = (double)n;
    double m = c / nd;
    double v = d / nd - m * m;
    double a = (double)I + m * (k - 1.0);
    if (a <= 0.0 || a * a <= (k * k * m * m * v) / (R * R))
        return 0;
    return 1;
}

/* (vi) Exact decision of I <= t for Sauvola with rational k = kn/kd >= 0 and
 * R = Rn/Rd > 0, from the Sec. 3.2 square-root-free form multiplied through
 * by n^2*kd*Rn > 0 (with s = sqrt(V)/n):
 *     A = kd*Rn*n^2*I + Rn*n*S1*(kn - kd),  B = kn*Rd*S1 >= 0,
 *     I <= t  <=>  A <= 0  or  A^2 <= B^2*V.
 * Integer arithmetic in 128 bits; returns the bit (0 when I <= t). */
uint8_t oracle_sauvola_bit_exact(uint32_t I, uint32_t S1, uint64_t S2,
                                 uint32_t n, int64_t kn, int64_t kd,
                                 int64_t Rn, int64_t Rd)
{
    __int128 V = (__int128)variance_numerator(S1, S2, n);
    __int128 nn = (__int128)n;
    __int128 A = (__int128)kd * Rn * nn * nn * (__int128)I +
                 (__int128)Rn * nn * (__int128)S1 * (__int128)(kn - kd);
    __int128 B = (__int128)kn * Rd * (__int128)S1;
    if (A <= 0)
        return 0;
    if (A * A <= B * B * V)
        return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* (vii) Packer: LSB-first, padding bits zero.                                */
/* ------------------------------------------------------------------------ */
void oracle_pack_bits(const uint8_t *bits, int64_t H, int64_t W, uint8_t *out,
                      int64_t out_pitch)
{
    for (int64_t i = 0; i < H; i++) {
        memset(out + i * out_pitch, 0, (size_t)out_pitch);
        for (int64_t j = 0; j < W; j++)
            if (bits[i * W + j])
                out[i * out_pitch + (j >> 3)] |= (uint8_t)(1u << (j & 7));
    }
}

/* ------------------------------------------------------------------------ */
/* Full binarizations: recursive sums (iii) + canonical threshold (v).        */
/* bits: H*W unpacked 0/1 bytes (may be NULL); out: packed (may be NULL).    */
/* ------------------------------------------------------------------------ */
static void threshold_row(int32_t method, const uint8_t *imgrow, int64_t W,
                          const uint32_t *S1, const uint64_t *S2,
                          const uint32_t *n, double k, double R, uint8_t *bits)
{
    for (int64_t j = 0; j < W; j++)
        bits[j] = decide(imgrow[j], oracle_threshold(method, S1[j], S2[j], n[j], k, R));
}

int oracle_binarize(int32_t method, const uint8_t *img, int64_t H, int64_t W,
                    int64_t pitch, int32_t h, int32_t w, double k, double R,
                    uint8_t *bits, uint8_t *out, int64_t out_pitch)
{
    if (check_args(H, W, pitch, h, w))
        return 1;
    if (out && out_pitch < (W + 7) / 8)
        return 1;
    size_t HW = (size_t)(H * W);
    uint32_t *S1 = (uint32_t *)malloc(HW * sizeof(uint32_t));
    uint64_t *S2 = (uint64_t *)malloc(HW * sizeof(uint64_t));
    uint32_t *n = (uint32_t *)malloc(HW * sizeof(uint32_t));
    uint8_t *b = bits ? bits : (uint8_t *)malloc(HW);
    if (!S1 || !S2 || !n || !b) {
        free(S1);
        free(S2);
        free(n);
        if (!bits)
            free(b);
        return 2;
    }
    oracle_window_sums_recursive(img, H, W, pitch, h, w, S1, S2, n);
    for (int64_t i = 0; i < H; i++)
        threshold_row(method, img + i * pitch, W, S1 + i * W, S2 + i * W,
                      n + i * W, k, R, b + i * W);
    if (out)
        oracle_pack_bits(b, H, W, out, out_pitch);
    free(S1);
    free(S2);
    free(n);
    if (!bits)
        free(b);
    return 0;
}

/* FP32 evaluation of the same canonical formula from the same exact
 * integers (the fast-path reading): returns the FP32 threshold. */
float oracle_threshold_f32(int32_t method, uint32_t S1, uint64_t S2, uint32_t n,
                           float k, float R)
{
    int64_t V = variance_numerator(S1, S2, n);
    float nd = (float)n;
    float m = (float)S1 / nd;
    float s = sqrtf((float)V / (nd * nd));
    if (method == ORACLE_SAUVOLA)
        return m * (1.0f + k * (s / R - 1.0f));
    return m + k * s;
}

/* ------------------------------------------------------------------------ */
/* (viii) Row-band parallel version of (iii)+(v), for timing only.  Each band  */
/* of rows restarts the stripe sums from its own warm-up rows, so bands are  */
/* independent; the result is identical to oracle_binarize.                  */
/* ------------------------------------------------------------------------ */
int oracle_binarize_parallel(int32_t method, const uint8_t *img, int64_t H,
                             int64_t W, int64_t pitch, int32_t h, int32_t w,
                             double k, double R, uint8_t *out, int64_t out_pitch,
                             int32_t nthreads)
{
    if (check_args(H, W, pitch, h, w) || out_pitch < (W + 7) / 8)
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    int nt = nthreads > 0 ? nthreads : 1;
    int64_t band = (H + nt - 1) / nt;
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static, 1) reduction(| : err)
#endif
    for (int64_t bi = 0; bi < nt; bi++) {
        int64_t i0 = bi * band, i1 = i0 + band < H ? i0 + band : H;
        if (i0 >= i1)
            continue;
        stripe_state st;
        st.H = H;
        st.W = W;
        st.pitch = pitch;
        st.img = img;
        st.l = l;
        st.r = r;
        st.o = o;
        st.u = u;
        st.C = (uint32_t *)malloc((size_t)W * sizeof(uint32_t));
        st.D = (uint32_t *)malloc((size_t)W * sizeof(uint32_t));
        uint32_t *S1 = (uint32_t *)malloc((size_t)W * sizeof(uint32_t));
        uint64_t *S2 = (uint64_t *)malloc((size_t)W * sizeof(uint64_t));
        uint32_t *nn = (uint32_t *)malloc((size_t)W * sizeof(uint32_t));
        uint8_t *bits = (uint8_t *)malloc((size_t)W);
        if (!st.C || !st.D || !S1 || !S2 || !nn || !bits) {
            err |= 1;
        } else {
            /* column sums over rows (i0-1-o, i0-1+u] = [i0-o, i0-o+h), the
               state just before row i0 */
            stripe_init(&st, i0 - o, (int64_t)h);
            for (int64_t i = i0; i < i1; i++) {
                stripe_advance(&st, i);
                window_row(&st, i, S1, S2, nn);
                threshold_row(method, img + i * pitch, W, S1, S2, nn, k, R, bits);
                uint8_t *orow = out + i * out_pitch;
                memset(orow, 0, (size_t)out_pitch);
                for (int64_t j = 0; j < W; j++)
                    if (bits[j])
                        orow[j >> 3] |= (uint8_t)(1u << (j & 7));
            }
        }
        free(st.C);
        free(st.D);
        free(S1);
        free(S2);
        free(nn);
        free(bits);
    }
    return err ? 2 : 0;
}

int32_t oracle_openmp_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Local quantile (Sec. 3.4): Q = rho-th smallest gray level of the clipped  */
/* window, rho = max(1, ceil(n*q_num/q_den)) in integers; t = Q - offset;     */
/* bit = 0 iff I <= t.                                                        */
/* ------------------------------------------------------------------------ */
static inline int64_t quantile_rank(uint32_t n, int32_t q_num, int32_t q_den)
{
    int64_t rho = ((int64_t)n * q_num + q_den - 1) / q_den;
    if (rho < 1)
        rho = 1;
    if (rho > (int64_t)n)
        rho = n;
    return rho;
}

static int check_q(int32_t q_num, int32_t q_den)
{
    return (q_den < 1 || q_num < 0 || q_num > q_den);
}

static int cmp_u8(const void *a, const void *b)
{
    return (int)*(const uint8_t *)a - (int)*(const uint8_t *)b;
}

/* (i') brute force: sort the window and index it. */
int oracle_window_quantile_sort(const uint8_t *img, int64_t H, int64_t W,
                                int64_t pitch, int32_t h, int32_t w,
                                int32_t q_num, int32_t q_den, uint8_t *Q)
{
    if (check_args(H, W, pitch, h, w) || check_q(q_num, q_den))
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    uint8_t *buf = (uint8_t *)malloc((size_t)h * (size_t)w);
    if (!buf)
        return 2;
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            size_t cnt = 0;
            for (int64_t a = i - o + 1; a <= i + u; a++)
                for (int64_t b = j - l + 1; b <= j + r; b++)
                    if (a >= 0 && a < H && b >= 0 && b < W)
                        buf[cnt++] = img[a * pitch + b];
            qsort(buf, cnt, 1, cmp_u8);
            Q[i * W + j] = buf[quantile_rank((uint32_t)cnt, q_num, q_den) - 1];
        }
    }
    free(buf);
    return 0;
}

/* Rank selection in a 256-bin histogram: smallest g with cum(g) >= rho. */
static inline uint8_t hist_select(const uint32_t *hist, int64_t rho)
{
    int64_t cum = 0;
    for (int g = 0; g < 256; g++) {
        cum += hist[g];
        if (cum >= rho)
            return (uint8_t)g;
    }
    return 255;
}

/* (i'') brute force by a 256-bin count of the window. */
int oracle_window_quantile_count(const uint8_t *img, int64_t H, int64_t W,
                                 int64_t pitch, int32_t h, int32_t w,
                                 int32_t q_num, int32_t q_den, uint8_t *Q)
{
    if (check_args(H, W, pitch, h, w) || check_q(q_num, q_den))
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    uint32_t hist[256];
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            memset(hist, 0, sizeof hist);
            uint32_t cnt = 0;
            for (int64_t a = i - o + 1; a <= i + u; a++)
                for (int64_t b = j - l + 1; b <= j + r; b++)
                    if (a >= 0 && a < H && b >= 0 && b < W) {
                        hist[img[a * pitch + b]]++;
                        cnt++;
                    }
            Q[i * W + j] = hist_select(hist, quantile_rank(cnt, q_num, q_den));
        }
    }
    return 0;
}

/* (iv) Sliding histogram (Sec. 3.4): along each row the window histogram is
 * updated by adding column j+r and removing column j-l (each restricted to
 * the window rows); Theta(HW*h) updates plus a 256-bin rank scan per pixel.
 * Rows are independent, so they may run in parallel (nthreads). */
int oracle_window_quantile_sliding(const uint8_t *img, int64_t H, int64_t W,
                                   int64_t pitch, int32_t h, int32_t w,
                                   int32_t q_num, int32_t q_den, uint8_t *Q,
                                   int32_t nthreads)
{
    if (check_args(H, W, pitch, h, w) || check_q(q_num, q_den))
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    int nt = nthreads > 0 ? nthreads : 1;
    (void)nt;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
#endif
    for (int64_t i = 0; i < H; i++) {
        uint32_t hist[256];
        memset(hist, 0, sizeof hist);
        int64_t a0 = i - o + 1 < 0 ? 0 : i - o + 1;
        int64_t a1 = i + u > H - 1 ? H - 1 : i + u;
        int64_t rows = a1 - a0 + 1;
        /* columns [0, r) enter before the first output column */
        for (int64_t b = 0; b < r && b < W; b++)
            for (int64_t a = a0; a <= a1; a++)
                hist[img[a * pitch + b]]++;
        for (int64_t j = 0; j < W; j++) {
            int64_t bin = j + r, bout = j - l;
            if (bin < W)
                for (int64_t a = a0; a <= a1; a++)
                    hist[img[a * pitch + bin]]++;
            if (bout >= 0)
                for (int64_t a = a0; a <= a1; a++)
                    hist[img[a * pitch + bout]]--;
            int64_t c0 = j - l + 1 < 0 ? 0 : j - l + 1;
            int64_t c1 = j + r > W - 1 ? W - 1 : j + r;
            uint32_t cnt = (uint32_t)(rows * (c1 - c0 + 1));
            Q[i * W + j] = hist_select(hist, quantile_rank(cnt, q_num, q_den));
        }
    }
    return 0;
}

/* Quantile binarization: bit = 0 iff I <= Q - offset (integers). */
int oracle_binarize_quantile(const uint8_t *img, int64_t H, int64_t W,
                             int64_t pitch, int32_t h, int32_t w, int32_t q_num,
                             int32_t q_den, int32_t offset, uint8_t *bits,
                             uint8_t *out, int64_t out_pitch, int32_t nthreads)
{
    if (check_args(H, W, pitch, h, w) || check_q(q_num, q_den))
        return 1;
    if (out && out_pitch < (W + 7) / 8)
        return 1;
    size_t HW = (size_t)(H * W);
    uint8_t *Q = (uint8_t *)malloc(HW);
    uint8_t *b = bits ? bits : (uint8_t *)malloc(HW);
    if (!Q || !b) {
        free(Q);
        if (!bits)
            free(b);
        return 2;
    }
    oracle_window_quantile_sliding(img, H, W, pitch, h, w, q_num, q_den, Q, nthreads);
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            int64_t t = (int64_t)Q[i * W + j] - offset;
            b[i * W + j] = ((int64_t)img[i * pitch + j] <= t) ? 0 : 1;
        }
    if (out)
        oracle_pack_bits(b, H, W, out, out_pitch);
    free(Q);
    if (!bits)
        free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Array forms of the per-pixel rules above (for the Python test harness).    */
/* img is the matching gray level of each element.                           */
/* ------------------------------------------------------------------------ */
void oracle_threshold_array(int32_t method, const uint32_t *S1, const uint64_t *S2,
                            const uint32_t *n, int64_t count, double k, double R,
                            double *t)
{
    for (int64_t q = 0; q < count; q++)
        t[q] = oracle_threshold(method, S1[q], S2[q], n[q], k, R);
}

void oracle_threshold_f32_array(int32_t method, const uint32_t *S1, const uint64_t *S2,
                                const uint32_t *n, int64_t count, float k, float R,
                                float *t)
{
    for (int64_t q = 0; q < count; q++)
        t[q] = oracle_threshold_f32(method, S1[q], S2[q], n[q], k, R);
}

void oracle_sauvola_bits_exact_array(const uint8_t *img, const uint32_t *S1,
                                     const uint64_t *S2, const uint32_t *n,
                                     int64_t count, int64_t kn, int64_t kd,
                                     int64_t Rn, int64_t Rd, uint8_t *bits)
{
    for (int64_t q = 0; q < count; q++)
        bits[q] = oracle_sauvola_bit_exact(img[q], S1[q], S2[q], n[q], kn, kd, Rn, Rd);
}

void oracle_sauvola_bits_paper_order_array(const uint8_t *img, const uint32_t *S1,
                                           const uint64_t *S2, const uint32_t *n,
                                           int64_t count, double k, double R,
                                           uint8_t *bits)
{
    for (int64_t q = 0; q < count; q++)
        bits[q] = oracle_sauvola_bit_paper_order(img[q], S1[q], S2[q], n[q], k, R);
}

/* Window sums of single pixels (i,j), straight from the definition: used to
 * check full-size outputs at sampled positions. */
void oracle_window_sums_at(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                           int32_t h, int32_t w, const int64_t *ii,
                           const int64_t *jj, int64_t count, uint32_t *S1,
                           uint64_t *S2, uint32_t *n)
{
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t q = 0; q < count; q++) {
        int64_t i = ii[q], j = jj[q];
        uint64_t s1 = 0, s2 = 0, cnt = 0;
        for (int64_t a = i - o + 1; a <= i + u; a++)
            for (int64_t b = j - l + 1; b <= j + r; b++)
                if (a >= 0 && a < H && b >= 0 && b < W) {
                    uint64_t v = img[a * pitch + b];
                    s1 += v;
                    s2 += v * v;
                    cnt++;
                }
        S1[q] = (uint32_t)s1;
        S2[q] = s2;
        n[q] = (uint32_t)cnt;
    }
}

/* Window quantile of single pixels by a 256-bin count. */
void oracle_window_quantile_at(const uint8_t *img, int64_t H, int64_t W,
                               int64_t pitch, int32_t h, int32_t w, int32_t q_num,
                               int32_t q_den, const int64_t *ii, const int64_t *jj,
                               int64_t count, uint8_t *Q)
{
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    uint32_t hist[256];
    for (int64_t q = 0; q < count; q++) {
        int64_t i = ii[q], j = jj[q];
        memset(hist, 0, sizeof hist);
        uint32_t cnt = 0;
        for (int64_t a = i - o + 1; a <= i + u; a++)
            for (int64_t b = j - l + 1; b <= j + r; b++)
                if (a >= 0 && a < H && b >= 0 && b < W) {
                    hist[img[a * pitch + b]]++;
                    cnt++;
                }
        Q[q] = hist_select(hist, quantile_rank(cnt, q_num, q_den));
    }
}

/* ------------------------------------------------------------------------ */
/* (ix) The other Table 1 methods (Wolf, Feng, Rais, Khurshid's NICK,         */
/*      Phansalkar): each keeps Algorithm 1's window statistics and changes   */
/*      only the threshold (Sec. 3.4).  Three of them also use the global     */
/*      minimum L, mean M and standard deviation S of the whole image         */
/*      (Table 1 notations).                                                  */
/* ------------------------------------------------------------------------ */

/* Global statistics by plain loops: L = min I, M = sum/N and
 * S = sqrt(Vg / (N*N)) with the exact numerator Vg = N*sumsq - sum^2
 * (population standard deviation, as the local s).  Vg needs 128 bits; its
 * conversion to double is the C conversion, round to nearest. */
int oracle_global_stats(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                        double *stats, uint64_t *sums)
{
    if (H < 1 || W < 1 || pitch < W)
        return 1;
    uint32_t L = 255;
    uint64_t sum = 0, sumsq = 0;
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            uint32_t v = img[i * pitch + j];
            L = v < L ? v : L;
            sum += v;
            sumsq += (uint64_t)v * v;
        }
    uint64_t N = (uint64_t)H * (uint64_t)W;
    unsigned __int128 Vg = (unsigned __int128)N * sumsq - (unsigned __int128)sum * sum;
    double Nd = (double)N;
    stats[0] = (double)L;
    stats[1] = (double)sum / Nd;
    stats[2] = sqrt((double)Vg / (Nd * Nd));
    if (sums) {
        sums[0] = sum;
        sums[1] = sumsq;
        sums[2] = N;
    }
    return 0;
}

/* Canonical FP64 thresholds of Table 1, one operation at a time, in this
 * order (m and s as in oracle_threshold; L, M, S from oracle_global_stats;
 * prm = {k, R, alpha1, k1, k2, gamma, p, q}):
 *   Wolf        t = m - (k*(m - L)) * (1 - s/R)
 *   Feng        x = s/R;  t = (alpha1*m + (k1*pow(x, 1+gamma))*(m - L))
 *                             + (k2*pow(x, gamma))*L
 *   Rais        d = max(m*s, M*S);  f = d > 0 ? (m*s - M*S)/d : 0;
 *               t = m + (k*f)*s
 *   NICK        t = m + k*sqrt(V/(n*n) + (m*m)*((n - 1)/n))
 *               (Table 1 writes hw; the clipped count n takes its place at
 *               the border, as it does in m and s)
 *   Phansalkar  t = m * ((1 + p*exp(-(q*m))) + k*(s/R - 1))
 * Sauvola and Niblack are oracle_threshold. */
double oracle_threshold_ext(int32_t method, uint32_t S1, uint64_t S2, uint32_t n,
                            const double *prm, const double *glob)
{
    const double k = prm[0], R = prm[1];
    if (method == ORACLE_SAUVOLA || method == ORACLE_NIBLACK)
        return oracle_threshold(method, S1, S2, n, k, R);
    int64_t V = variance_numerator(S1, S2, n);
    double nd = (double)n;
    double m = (double)S1 / nd;
    double v = (double)V / (nd * nd);
    double s = sqrt(v);
    double L = glob[0], M = glob[1], S = glob[2];
    switch (method) {
    case ORACLE_WOLF:
        return m - (k * (m - L)) * (1.0 - s / R);
    case ORACLE_FENG: {
        double alpha1 = prm[2], k1 = prm[3], k2 = prm[4], gamma = prm[5];
        double x = s / R;
        double a = alpha1 * m;
        double b = (k1 * pow(x, 1.0 + gamma)) * (m - L);
        double c = (k2 * pow(x, gamma)) * L;
        return (a + b) + c;
    }
    case ORACLE_RAIS: {
        double ms = m * s, MS = M * S;
        double d = ms > MS ? ms : MS;
        double f = d > 0.0 ? (ms - MS) / d : 0.0;
        return m + (k * f) * s;
    }
    case ORACLE_NICK:
        return m + k * sqrt(v + (m * m) * ((nd - 1.0) / nd));
    case ORACLE_PHANSALKAR: {
        double p = prm[6], q = prm[7];
        return m * ((1.0 + p * exp(-(q * m))) + k * (s / R - 1.0));
    }
    default:
        return NAN;
    }
}

void oracle_threshold_ext_array(int32_t method, const uint32_t *S1, const uint64_t *S2,
                                const uint32_t *n, int64_t count, const double *prm,
                                const double *glob, double *t)
{
    for (int64_t x = 0; x < count; x++)
        t[x] = oracle_threshold_ext(method, S1[x], S2[x], n[x], prm, glob);
}

/* Full binarization with any Table 1 method: global statistics, Algorithm 1
 * window sums, canonical threshold, I <= t -> 0. */
int oracle_binarize_ext(int32_t method, const uint8_t *img, int64_t H, int64_t W,
                        int64_t pitch, int32_t h, int32_t w, const double *prm,
                        uint8_t *bits, uint8_t *out, int64_t out_pitch)
{
    if (check_args(H, W, pitch, h, w) || method < 0 || method > ORACLE_PHANSALKAR ||
        method == 2)
        return 1;
    if (out && out_pitch < (W + 7) / 8)
        return 1;
    double glob[3];
    oracle_global_stats(img, H, W, pitch, glob, NULL);
    size_t HW = (size_t)(H * W);
    uint32_t *S1 = (uint32_t *)malloc(HW * sizeof(uint32_t));
    uint64_t *S2 = (uint64_t *)malloc(HW * sizeof(uint64_t));
    uint32_t *n = (uint32_t *)malloc(HW * sizeof(uint32_t));
    uint8_t *b = bits ? bits : (uint8_t *)malloc(HW);
    if (!S1 || !S2 || !n || !b) {
        free(S1);
        free(S2);
        free(n);
        if (!bits)
            free(b);
        return 2;
    }
    oracle_window_sums_recursive(img, H, W, pitch, h, w, S1, S2, n);
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            int64_t x = i * W + j;
            b[x] = decide(img[i * pitch + j],
                          oracle_threshold_ext(method, S1[x], S2[x], n[x], prm, glob));
        }
    if (out)
        oracle_pack_bits(b, H, W, out, out_pitch);
    free(S1);
    free(S2);
    free(n);
    if (!bits)
        free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (x) Local minimum and maximum (Sec. 3.4: Bernsen's midrange and the local  */
/*     contrast, computed recursively with deques).  The window is Algorithm  */
/*     1's, clipped to the image: out-of-image pixels take no part (a 0 would */
/*     be a false minimum).  The window always holds its own centre pixel.    */
/* ------------------------------------------------------------------------ */

/* Definition: direct loops over the clipped window. */
int oracle_window_minmax_bruteforce(const uint8_t *img, int64_t H, int64_t W,
                                    int64_t pitch, int32_t h, int32_t w,
                                    uint8_t *mn, uint8_t *mx)
{
    if (check_args(H, W, pitch, h, w))
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            uint32_t lo = 255, hi = 0;
            for (int64_t a = i - o + 1; a <= i + u; a++)
                for (int64_t b = j - l + 1; b <= j + r; b++) {
                    if (a < 0 || a >= H || b < 0 || b >= W)
                        continue;
                    uint32_t v = img[a * pitch + b];
                    lo = v < lo ? v : lo;
                    hi = v > hi ? v : hi;
                }
            mn[i * W + j] = (uint8_t)lo;
            mx[i * W + j] = (uint8_t)hi;
        }
    return 0;
}

/* Sliding extremum of one line of `len` values (stride `step`) over the
 * window (x - back, x + fwd] clipped to [0, len), with a monotonic deque of
 * indices: each index enters once and leaves once, so Theta(len) for any
 * window (the recursive scheme Sec. 3.4 names).  want_max selects max. */
static void slide_extremum(const uint8_t *src, int64_t step, int64_t len,
                           int32_t back, int32_t fwd, int want_max,
                           uint8_t *dst, int64_t dstep, int64_t *dq)
{
    int64_t head = 0, tail = 0; /* deque dq[head, tail) */
    int64_t next = 0;           /* next index to enter */
    for (int64_t x = 0; x < len; x++) {
        int64_t last = x + fwd < len - 1 ? x + fwd : len - 1;
        while (next <= last) {
            uint8_t v = src[next * step];
            while (tail > head) {
                uint8_t b = src[dq[tail - 1] * step];
                if (want_max ? (b <= v) : (b >= v))
                    tail--;
                else
                    break;
            }
            dq[tail++] = next++;
        }
        while (dq[head] <= x - back)
            head++;
        dst[x * dstep] = src[dq[head] * step];
    }
}

/* Separable sliding min/max: vertical extrema of every column over rows
 * (i-o, i+u], then horizontal extrema of those over columns (j-l, j+r]. */
int oracle_window_minmax_deque(const uint8_t *img, int64_t H, int64_t W,
                               int64_t pitch, int32_t h, int32_t w,
                               uint8_t *mn, uint8_t *mx)
{
    if (check_args(H, W, pitch, h, w))
        return 1;
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    size_t HW = (size_t)(H * W);
    uint8_t *vmn = (uint8_t *)malloc(HW), *vmx = (uint8_t *)malloc(HW);
    int64_t *dq = (int64_t *)malloc((size_t)(H > W ? H : W) * sizeof(int64_t));
    if (!vmn || !vmx || !dq) {
        free(vmn);
        free(vmx);
        free(dq);
        return 2;
    }
    for (int64_t j = 0; j < W; j++) {
        slide_extremum(img + j, pitch, H, o, u, 0, vmn + j, W, dq);
        slide_extremum(img + j, pitch, H, o, u, 1, vmx + j, W, dq);
    }
    for (int64_t i = 0; i < H; i++) {
        slide_extremum(vmn + i * W, 1, W, l, r, 0, mn + i * W, 1, dq);
        slide_extremum(vmx + i * W, 1, W, l, r, 1, mx + i * W, 1, dq);
    }
    free(vmn);
    free(vmx);
    free(dq);
    return 0;
}

/* Bernsen's decision from the window extrema, in integers:
 *   contrast c = mx - mn;
 *   c >= contrast_limit:  bit = 0 iff I <= (mn + mx)/2, i.e. 2I <= mn + mx;
 *   c <  contrast_limit:  the window is one class, dark (0) iff its
 *                         midrange is at most 127.5, i.e. mn + mx <= 255. */
static inline uint8_t bernsen_bit(uint32_t I, uint32_t lo, uint32_t hi,
                                  int32_t contrast_limit)
{
    if ((int32_t)(hi - lo) >= contrast_limit)
        return (2 * I <= lo + hi) ? 0 : 1;
    return (lo + hi <= 255) ? 0 : 1;
}

int oracle_binarize_bernsen(const uint8_t *img, int64_t H, int64_t W,
                            int64_t pitch, int32_t h, int32_t w,
                            int32_t contrast_limit, uint8_t *bits,
                            uint8_t *out, int64_t out_pitch)
{
    if (check_args(H, W, pitch, h, w) || contrast_limit < 0 || contrast_limit > 256)
        return 1;
    if (out && out_pitch < (W + 7) / 8)
        return 1;
    size_t HW = (size_t)(H * W);
    uint8_t *mn = (uint8_t *)malloc(HW), *mx = (uint8_t *)malloc(HW);
    uint8_t *b = bits ? bits : (uint8_t *)malloc(HW);
    if (!mn || !mx || !b) {
        free(mn);
        free(mx);
        if (!bits)
            free(b);
        return 2;
    }
    int rc = oracle_window_minmax_deque(img, H, W, pitch, h, w, mn, mx);
    if (rc == 0) {
        for (int64_t i = 0; i < H; i++)
            for (int64_t j = 0; j < W; j++)
                b[i * W + j] = bernsen_bit(img[i * pitch + j], mn[i * W + j],
                                           mx[i * W + j], contrast_limit);
        if (out)
            oracle_pack_bits(b, H, W, out, out_pitch);
    }
    free(mn);
    free(mx);
    if (!bits)
        free(b);
    return rc;
}

/* Window extrema at sampled positions (direct loops), for full-size checks. */
void oracle_window_minmax_at(const uint8_t *img, int64_t H, int64_t W,
                             int64_t pitch, int32_t h, int32_t w,
                             const int64_t *ii, const int64_t *jj, int64_t count,
                             uint8_t *mn, uint8_t *mx)
{
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t x = 0; x < count; x++) {
        int64_t i = ii[x], j = jj[x];
        uint32_t lo = 255, hi = 0;
        for (int64_t a = i - o + 1; a <= i + u; a++)
            for (int64_t b = j - l + 1; b <= j + r; b++) {
                if (a < 0 || a >= H || b < 0 || b >= W)
                    continue;
                uint32_t v = img[a * pitch + b];
                lo = v < lo ? v : lo;
                hi = v > hi ? v : hi;
            }
        mn[x] = (uint8_t)lo;
        mx[x] = (uint8_t)hi;
    }
}

/* ------------------------------------------------------------------------ */
/* (xi) Haar-like features (Sec. 3.4: the recursive sums serve any sum over  */
/*      rectangles).  A feature is a sum over Algorithm 1's h x w window with */
/*      a separable, piecewise-constant weight f(a) g(b): the rows of the     */
/*      window are cut into n_row segments (length, weight), the columns into */
/*      n_col segments.  Two segments of opposite weight in one direction and */
/*      one in the other give Viola and Jones's two-rectangle features, three */
/*      give the three-rectangle ones, two by two the four-rectangle one.     */
/*      Out-of-image pixels are 0, as for the window sums.                    */
/* ------------------------------------------------------------------------ */
static int haar_profile(const int32_t *len, const int32_t *wt, int32_t nseg,
                        int32_t total, int32_t *prof)
{
    int32_t pos = 0;
    for (int32_t s = 0; s < nseg; s++) {
        if (len[s] < 1)
            return 1;
        for (int32_t q = 0; q < len[s]; q++) {
            if (pos >= total)
                return 1;
            prof[pos++] = wt[s];
        }
    }
    return pos == total ? 0 : 1;
}

/* Definition: the weighted sum over the window, by direct loops. */
int oracle_haar_bruteforce(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                           const int32_t *row_len, const int32_t *row_wt, int32_t n_row,
                           const int32_t *col_len, const int32_t *col_wt, int32_t n_col,
                           int32_t *out)
{
    int32_t h = 0, w = 0;
    for (int32_t s = 0; s < n_row; s++)
        h += row_len[s];
    for (int32_t s = 0; s < n_col; s++)
        w += col_len[s];
    if (check_args(H, W, pitch, h, w))
        return 1;
    int32_t *f = (int32_t *)malloc((size_t)h * sizeof(int32_t));
    int32_t *g = (int32_t *)malloc((size_t)w * sizeof(int32_t));
    if (!f || !g || haar_profile(row_len, row_wt, n_row, h, f) ||
        haar_profile(col_len, col_wt, n_col, w, g)) {
        free(f);
        free(g);
        return 1;
    }
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            int64_t acc = 0;
            for (int32_t a = 0; a < h; a++)
                for (int32_t b = 0; b < w; b++)
                    acc += (int64_t)f[a] * g[b] *
                           (int64_t)px(img, H, W, pitch, i - o + 1 + a, j - l + 1 + b);
            out[i * W + j] = (int32_t)acc;
        }
    free(f);
    free(g);
    return 0;
}

/* Viola and Jones's route: every rectangle (row segment x column segment)
 * summed by four lookups in the Sec. 2 integral image, times the product of
 * the two weights. */
int oracle_haar_integral(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                         const int32_t *row_len, const int32_t *row_wt, int32_t n_row,
                         const int32_t *col_len, const int32_t *col_wt, int32_t n_col,
                         int32_t *out)
{
    int32_t h = 0, w = 0;
    for (int32_t s = 0; s < n_row; s++)
        h += row_len[s];
    for (int32_t s = 0; s < n_col; s++)
        w += col_len[s];
    if (check_args(H, W, pitch, h, w) || n_row < 1 || n_col < 1)
        return 1;
    for (int32_t s = 0; s < n_row; s++)
        if (row_len[s] < 1)
            return 1;
    for (int32_t s = 0; s < n_col; s++)
        if (col_len[s] < 1)
            return 1;
    int64_t *J = (int64_t *)malloc((size_t)(H * W) * sizeof(int64_t));
    if (!J)
        return 2;
    for (int64_t i = 0; i < H; i++) {
        int64_t rowsum = 0;
        for (int64_t j = 0; j < W; j++) {
            rowsum += img[i * pitch + j];
            J[i * W + j] = rowsum + (i > 0 ? J[(i - 1) * W + j] : 0);
        }
    }
    int32_t l, r, o, u;
    oracle_window_params(h, w, &l, &r, &o, &u);
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            int64_t acc = 0, a0 = i - o; /* rows (a0 + start, a0 + end] */
            int32_t rs = 0;
            for (int32_t p = 0; p < n_row; p++) {
                int32_t cs = 0;
                for (int32_t q = 0; q < n_col; q++) {
                    /* rows (i-o+rs, i-o+rs+len], columns (j-l+cs, j-l+cs+len] */
                    int64_t r0 = a0 + rs, r1 = a0 + rs + row_len[p];
                    int64_t c0 = j - l + cs, c1 = j - l + cs + col_len[q];
                    int64_t s = J_at(J, H, W, r1, c1) - J_at(J, H, W, r0, c1) -
                                J_at(J, H, W, r1, c0) + J_at(J, H, W, r0, c0);
                    acc += (int64_t)row_wt[p] * col_wt[q] * s;
                    cs += col_len[q];
                }
                rs += row_len[p];
            }
            out[i * W + j] = (int32_t)acc;
        }
    free(J);
    return 0;
}
