// The other thresholds of Table 1 (Wolf, Feng, Rais, NICK, Phansalkar) on
// the same window statistics, and the global statistics L, M, S (Table 1
// notations) that three of them use.  Included by bz_window.cuh after the
// Sauvola/Niblack threshold helpers.
#pragma once

namespace bz {

enum Method : int {
    METHOD_SAUVOLA = 0,
    METHOD_NIBLACK = 1,
    METHOD_QUANTILE = 2,
    METHOD_WOLF = 3,
    METHOD_FENG = 4,
    METHOD_RAIS = 5,
    METHOD_NICK = 6,
    METHOD_PHANSALKAR = 7,
};

// Exact image-wide sums, produced by k_global_stats from an all-zero start:
// the minimum is kept as Linv = 255 - L, a maximum, so that one memset
// initialises everything.
struct GStats {
    unsigned int Linv;
    unsigned int pad;
    unsigned long long sum, sumsq;
};

// Global minimum, mean and population standard deviation in FP64.
struct Global {
    double L, M, S;
};

// Round-to-nearest-even conversion of the 128-bit unsigned integer hi:lo to
// binary64 (IEEE 754 rounding of the value's leading 53 bits, with the bits
// below them folded into a round bit and a sticky bit).
__device__ __forceinline__ double u128_to_double_rn(unsigned long long hi, unsigned long long lo)
{
    if (hi == 0ull)
        return __ull2double_rn(lo);
    const int sh = 64 - __clzll((long long)hi);  // significant bits of hi, 1..64
    const unsigned long long top = sh == 64 ? hi : (hi << (64 - sh)) | (lo >> sh);
    const bool sticky = sh == 64 ? lo != 0ull : (lo << (64 - sh)) != 0ull;
    unsigned long long mant = top >> 11;  // 53 bits, leading bit set
    const unsigned long long rem = top & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (sticky || (mant & 1ull))))
        mant += 1ull;  // may become 2^53: still exact
    return ldexp(__ull2double_rn(mant), 11 + sh);
}

// L, M = sum/N and S = sqrt(Vg/(N*N)) with the exact numerator
// Vg = N*sumsq - sum^2 (>= 0), evaluated in this order.
__device__ __forceinline__ Global global_lms(const GStats &G, unsigned long long N)
{
    Global r;
    r.L = __uint2double_rn(255u - G.Linv);
    const double Nd = __ull2double_rn(N);
    r.M = __ddiv_rn(__ull2double_rn(G.sum), Nd);
    const unsigned long long ph = __umul64hi(N, G.sumsq), pl = N * G.sumsq;
    const unsigned long long qh = __umul64hi(G.sum, G.sum), ql = G.sum * G.sum;
    const unsigned long long vl = pl - ql;
    const unsigned long long vh = ph - qh - (pl < ql ? 1ull : 0ull);
    r.S = __dsqrt_rn(__ddiv_rn(u128_to_double_rn(vh, vl), __dmul_rn(Nd, Nd)));
    return r;
}

// Parameters of the Table 1 thresholds beyond k and R.
struct ExtParams {
    double alpha1, k1, k2, gamma;  // Feng
    double p, q;                   // Phansalkar
};

// Canonical FP64 thresholds, one rounded operation at a time in the order
//   Wolf        t = m - (k*(m - L)) * (1 - s/R)
//   Feng        x = s/R;  t = (alpha1*m + (k1*x^(1+gamma))*(m - L)) + (k2*x^gamma)*L
//   Rais        d = max(m*s, M*S);  f = d > 0 ? (m*s - M*S)/d : 0;  t = m + (k*f)*s
//   NICK        t = m + k*sqrt(V/(n*n) + (m*m)*((n - 1)/n))
//   Phansalkar  t = m * ((1 + p*exp(-(q*m))) + k*(s/R - 1))
// with nd = n, m = S1/nd, v = V/(nd*nd), s = sqrt(v) as for Sauvola.  NICK's
// hw of Table 1 is the clipped count n at the border, as in m and s.
__device__ __forceinline__ double canonical_t_ext(int method, uint32_t S1, uint64_t S2, uint32_t n,
                                                  double k, double R, const ExtParams &X,
                                                  const Global &G)
{
    const long long V = (long long)n * (long long)S2 - (long long)S1 * (long long)S1;
    const double nd = __uint2double_rn(n);
    // V = 0: all in-image pixels of the window are equal, so the quotients
    // below are exact (m = S1 / n, v = s = +0) and need no FP64 division
    const double m = V == 0 ? __uint2double_rn(S1 / n) : __ddiv_rn(__uint2double_rn(S1), nd);
    const double v = V == 0 ? 0.0 : __ddiv_rn(__ll2double_rn(V), __dmul_rn(nd, nd));
    const double s = V == 0 ? 0.0 : __dsqrt_rn(v);
    switch (method) {
    case METHOD_WOLF:
        return __dadd_rn(m, -__dmul_rn(__dmul_rn(k, __dadd_rn(m, -G.L)),
                                       __dadd_rn(1.0, -__ddiv_rn(s, R))));
    case METHOD_FENG: {
        const double x = __ddiv_rn(s, R);
        const double a = __dmul_rn(X.alpha1, m);
        const double b = __dmul_rn(__dmul_rn(X.k1, pow(x, __dadd_rn(1.0, X.gamma))), __dadd_rn(m, -G.L));
        const double c = __dmul_rn(__dmul_rn(X.k2, pow(x, X.gamma)), G.L);
        return __dadd_rn(__dadd_rn(a, b), c);
    }
    case METHOD_RAIS: {
        const double ms = __dmul_rn(m, s), MS = __dmul_rn(G.M, G.S);
        const double d = ms > MS ? ms : MS;
        const double f = d > 0.0 ? __ddiv_rn(__dadd_rn(ms, -MS), d) : 0.0;
        return __dadd_rn(m, __dmul_rn(__dmul_rn(k, f), s));
    }
    case METHOD_NICK:
        return __dadd_rn(m, __dmul_rn(k, __dsqrt_rn(__dadd_rn(
                                             v, __dmul_rn(__dmul_rn(m, m),
                                                          __ddiv_rn(__dadd_rn(nd, -1.0), nd))))));
    default: {  // METHOD_PHANSALKAR
        const double e = exp(-__dmul_rn(X.q, m));
        return __dmul_rn(m, __dadd_rn(__dadd_rn(1.0, __dmul_rn(X.p, e)),
                                      __dmul_rn(k, __dadd_rn(__ddiv_rn(s, R), -1.0))));
    }
    }
}

// FP32 constants of one launch, derived per tile from the parameters and
// the global statistics.
struct ExtF {
    float c0, c1, c2;  // method-specific coefficients (see ext_t32)
    float L, MS, invR, gamma, q;
    float eps;
};

__device__ __forceinline__ ExtF make_extf(int method, double k, double R, const ExtParams &X,
                                          const Global &G, float eps)
{
    ExtF F;
    F.L = (float)G.L;
    F.MS = (float)(G.M * G.S);
    F.invR = (float)(1.0 / R);
    F.gamma = (float)X.gamma;
    F.q = (float)X.q;
    F.eps = eps;
    switch (method) {
    case METHOD_WOLF:  // t = (1-k) m + k L + (k/R)(m - L) s
        F.c0 = (float)(1.0 - k);
        F.c1 = (float)(k * G.L);
        F.c2 = (float)(k / R);
        break;
    case METHOD_FENG:  // t = alpha1 m + k1 x^(1+gamma) (m - L) + k2 x^gamma L
        F.c0 = (float)X.alpha1;
        F.c1 = (float)X.k1;
        F.c2 = (float)X.k2;
        break;
    case METHOD_PHANSALKAR:  // t = (1-k) m + p m e + (k/R) m s
        F.c0 = (float)(1.0 - k);
        F.c1 = (float)X.p;
        F.c2 = (float)(k / R);
        break;
    default:  // Rais, NICK: t = m + k (...)
        F.c0 = (float)k;
        F.c1 = 0.0f;
        F.c2 = 0.0f;
        break;
    }
    return F;
}

// FP32 threshold of a Table 1 method from mu = m and var = s^2, and a bound
// `bnd` on |t32 - t64|.  The bound is eps * mag, where mag adds up the
// absolute values of the terms with every difference replaced by a sum (so
// that cancellation cannot hide an error), plus the relative error rho of
// each transcendental factor times its term, plus a floor for FP32
// underflow.  eps covers the FP32 roundings (each input, the reciprocal of
// n, sqrt.approx, one operation per factor) and the FP64 formula's own error
// (far below 2^-40 relative).  For Feng and Phansalkar rho follows the
// accuracy that the CUDA math library documents (log2f 1 ulp, exp2f and expf
// 2 ulp) and the argument's propagated error (|z| times the relative error of
// the argument), with a factor of 4 to spare.
template <int METHOD>
__device__ __forceinline__ float ext_t32(const ExtF &F, float mu, float var, float inv_n,
                                         float &bnd)
{
    constexpr float u = 5.9604645e-8f;  // 2^-24
    constexpr float floor_abs = 1e-25f;
    if (METHOD == METHOD_WOLF) {
        const float s = sqrt_approx(var);
        const float t = fmaf(F.c2 * (mu - F.L), s, fmaf(F.c0, mu, F.c1));
        bnd = fmaf(F.eps, fmaf(fabsf(F.c2) * (mu + F.L), s, fmaf(fabsf(F.c0), mu, fabsf(F.c1))),
                   floor_abs);
        return t;
    } else if (METHOD == METHOD_FENG) {
        const float s = sqrt_approx(var);
        const float x = s * F.invR;
        float p0, z = 0.0f;
        if (x > 0.0f) {
            z = F.gamma * log2f(x);
            p0 = exp2f(z);
        } else {
            p0 = F.gamma == 0.0f ? 1.0f : 0.0f;
        }
        const float p1 = p0 * x;
        const float t = fmaf(F.c2 * p0, F.L, fmaf(F.c1 * p1, mu - F.L, F.c0 * mu));
        const float pw = fmaf(fabsf(F.c1) * p1, mu + F.L, fabsf(F.c2) * p0 * F.L);
        const float rho = u * fmaf(16.0f, fabsf(z), fmaf(32.0f, F.gamma, 32.0f));
        bnd = fmaf(F.eps, fmaf(fabsf(F.c0), mu, pw), fmaf(rho, pw, floor_abs));
        return t;
    } else if (METHOD == METHOD_RAIS) {
        const float s = sqrt_approx(var);
        const float ms = mu * s;
        const float den = fmaxf(ms, F.MS);
        const float f = den > 0.0f ? __fdiv_rn(ms - F.MS, den) : 0.0f;
        const float t = fmaf(F.c0 * f, s, mu);
        bnd = fmaf(F.eps, fmaf(3.0f * fabsf(F.c0), s, mu), floor_abs);
        return t;
    } else if (METHOD == METHOD_NICK) {
        const float sn = sqrt_approx(fmaf(mu * mu, 1.0f - inv_n, var));
        const float t = fmaf(F.c0, sn, mu);
        bnd = fmaf(F.eps, fmaf(fabsf(F.c0), sn, mu), floor_abs);
        return t;
    } else {  // METHOD_PHANSALKAR
        const float s = sqrt_approx(var);
        const float z = F.q * mu;
        const float e = expf(-z);
        const float pe = F.c1 * mu * e;
        const float t = fmaf(F.c2 * mu, s, fmaf(F.c0, mu, pe));
        const float ape = fabsf(pe);
        const float rho = u * fmaf(16.0f, z, 16.0f);
        bnd = fmaf(F.eps, fmaf(fabsf(F.c2) * mu, s, fmaf(fabsf(F.c0), mu, ape)),
                   fmaf(rho, ape, floor_abs));
        return t;
    }
}

}  // namespace bz
