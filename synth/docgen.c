/*
 * Seeded synthetic document images: the stand-in for the scanned, degraded
 * document pages (DIBCO-style) the binarization method is evaluated on.
 *
 * This module holds no binarization arithmetic; it only draws pixels.  Both
 * the CUDA library's tests/benchmark and the CPU oracle's tests take their
 * inputs from here.
 *
 * Determinism: only integer operations and the IEEE-754 basic operations
 * (+ - * / sqrt, each correctly rounded) are used, with FMA contraction off,
 * so the same seed gives the same bytes on x86-64 and on aarch64.
 *
 * Recipe (paint order):
 *   1. background 200 - 60*j/(W-1) (illumination gradient across the width);
 *   2. n_stains filled ellipses, centre uniform in the image, semi-axes
 *      uniform in [0.05, 0.2]*min(H,W), uniform rotation, value uniform
 *      integer in [120, 160];
 *   3. dark strokes of value 40, 2 px wide, length uniform in [8, 48] px,
 *      direction one of {0, 90, +45, -45 degrees, uniform}, painted until
 *      stroke pixels cover >= stroke_frac of the image;
 *   4. additive noise of standard deviation sigma (Irwin-Hall sum of four
 *      uniforms, scaled to unit variance), rounded half up, clipped to
 *      [0, 255];
 *   5. salt-and-pepper: each pixel set to 0 with probability sp/2 and to 255
 *      with probability sp/2.
 * PRNG: SplitMix64 (Steele, Lea, Flood 2014); uniform doubles take the top
 * 53 bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s;
} rng_t;

static inline uint64_t rng_next(rng_t *g)
{
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline double rng_unit(rng_t *g) /* [0, 1) */
{
    return (double)(rng_next(g) >> 11) * (1.0 / 9007199254740992.0);
}

static inline int64_t rng_int(rng_t *g, int64_t lo, int64_t hi) /* [lo, hi] */
{
    uint64_t span = (uint64_t)(hi - lo) + 1u;
    return lo + (int64_t)(rng_next(g) % span);
}

/* random direction (dx, dy) of unit length, by rejection in the unit disk */
static void rng_dir(rng_t *g, double *dx, double *dy)
{
    for (;;) {
        double x = 2.0 * rng_unit(g) - 1.0, y = 2.0 * rng_unit(g) - 1.0;
        double q = x * x + y * y;
        if (q > 1e-6 && q <= 1.0) {
            double L = sqrt(q);
            *dx = x / L;
            *dy = y / L;
            return;
        }
    }
}

static inline int64_t round_half_up(double x)
{
    return (int64_t)floor(x + 0.5);
}

/* Returns 0 on success.  img has H rows of `pitch` bytes; bytes between W
 * and pitch are set to 0. */
int synth_document(uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                   uint64_t seed, int32_t n_stains, double stroke_frac,
                   double sigma, double sp)
{
    if (H < 1 || W < 1 || pitch < W || sp < 0.0 || sp >= 1.0 || sigma < 0.0)
        return 1;
    rng_t g = {seed};
    /* work in 16-bit so noise can be added before clipping */
    int16_t *buf = (int16_t *)malloc((size_t)(H * W) * sizeof(int16_t));
    if (!buf)
        return 2;
    /* 1. background */
    for (int64_t j = 0; j < W; j++) {
        double v = W > 1 ? 200.0 - 60.0 * (double)j / (double)(W - 1) : 200.0;
        int16_t b = (int16_t)round_half_up(v);
        for (int64_t i = 0; i < H; i++)
            buf[i * W + j] = b;
    }
    /* 2. stains */
    double mn = (double)(H < W ? H : W);
    for (int32_t e = 0; e < n_stains; e++) {
        double cy = rng_unit(&g) * (double)H, cx = rng_unit(&g) * (double)W;
        double a = (0.05 + 0.15 * rng_unit(&g)) * mn;
        double b = (0.05 + 0.15 * rng_unit(&g)) * mn;
        double dx, dy;
        rng_dir(&g, &dx, &dy);
        int16_t val = (int16_t)rng_int(&g, 120, 160);
        double ext = a > b ? a : b;
        int64_t i0 = (int64_t)floor(cy - ext), i1 = (int64_t)ceil(cy + ext);
        int64_t j0 = (int64_t)floor(cx - ext), j1 = (int64_t)ceil(cx + ext);
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > H - 1) i1 = H - 1;
        if (j1 > W - 1) j1 = W - 1;
        for (int64_t i = i0; i <= i1; i++)
            for (int64_t j = j0; j <= j1; j++) {
                double y = (double)i + 0.5 - cy, x = (double)j + 0.5 - cx;
                double p = (x * dx + y * dy) / a, q = (y * dx - x * dy) / b;
                if (p * p + q * q <= 1.0)
                    buf[i * W + j] = val;
            }
    }
    /* 3. strokes */
    int64_t target = (int64_t)ceil(stroke_frac * (double)(H * W));
    int64_t painted = 0;
    const double rs2 = 0.70710678118654752440;
    int64_t guard = 0;
    while (painted < target && guard < 64 * (H * W + 64)) {
        double y0 = rng_unit(&g) * (double)H, x0 = rng_unit(&g) * (double)W;
        int64_t len = rng_int(&g, 8, 48);
        int64_t kind = rng_int(&g, 0, 4);
        double ux, uy;
        switch (kind) {
        case 0: ux = 1.0; uy = 0.0; break;
        case 1: ux = 0.0; uy = 1.0; break;
        case 2: ux = rs2; uy = rs2; break;
        case 3: ux = rs2; uy = -rs2; break;
        default: rng_dir(&g, &ux, &uy); break;
        }
        for (int64_t t = 0; t <= len; t++) {
            int64_t ci = round_half_up(y0 + (double)t * uy);
            int64_t cj = round_half_up(x0 + (double)t * ux);
            for (int64_t di = 0; di < 2; di++)
                for (int64_t dj = 0; dj < 2; dj++) {
                    int64_t i = ci + di, j = cj + dj;
                    guard++;
                    if (i < 0 || i >= H || j < 0 || j >= W)
                        continue;
                    if (buf[i * W + j] != 40) {
                        buf[i * W + j] = 40;
                        painted++;
                    }
                }
        }
    }
    /* 4. noise, rounding, clipping */
    const double scale = sigma * 1.7320508075688772935; /* sqrt(3) */
    for (int64_t i = 0; i < H; i++) {
        uint8_t *row = img + i * pitch;
        for (int64_t j = 0; j < W; j++) {
            double v = (double)buf[i * W + j];
            if (sigma > 0.0) {
                double s4 = rng_unit(&g) + rng_unit(&g) + rng_unit(&g) + rng_unit(&g);
                v = v + scale * (s4 - 2.0);
            }
            int64_t q = round_half_up(v);
            row[j] = (uint8_t)(q < 0 ? 0 : (q > 255 ? 255 : q));
        }
        if (pitch > W)
            memset(row + W, 0, (size_t)(pitch - W));
    }
    /* 5. salt and pepper */
    if (sp > 0.0) {
        uint64_t half = (uint64_t)(sp * 0.5 * 18446744073709551616.0);
        for (int64_t i = 0; i < H; i++)
            for (int64_t j = 0; j < W; j++) {
                uint64_t z = rng_next(&g);
                if (z < half)
                    img[i * pitch + j] = 0;
                else if (z < 2 * half)
                    img[i * pitch + j] = 255;
            }
    }
    free(buf);
    return 0;
}

/* Uniform random bytes (for adversarial parity cases). */
int synth_uniform(uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                  uint64_t seed, int32_t lo, int32_t hi)
{
    if (H < 1 || W < 1 || pitch < W || lo < 0 || hi > 255 || lo > hi)
        return 1;
    rng_t g = {seed};
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++)
            img[i * pitch + j] = (uint8_t)rng_int(&g, lo, hi);
        for (int64_t j = W; j < pitch; j++)
            img[i * pitch + j] = 0;
    }
    return 0;
}

/* Raw SplitMix64 stream (used by the Python side to draw workload shapes). */
void synth_splitmix64(uint64_t seed, uint64_t *out, int64_t count)
{
    rng_t g = {seed};
    for (int64_t k = 0; k < count; k++)
        out[k] = rng_next(&g);
}
