// FP64 elementary functions for the likelihood kernels, written for this GPU
// where the FP64 pipe issues 2 operations per clock per SM (64x fewer than
// FP32).  Each function uses a table lookup (shared memory) so that its
// polynomial is short, and integer operations for exponent handling; every
// value is computed in FP64 and accurate to a few units in the last place
// (the table generator and the limits are in gen_fp64_tables.py).
//
//   exp_fast(x)      2^(k/64) T_j (1 + p(r)), r = x - k ln2/64, |r| <= ln2/128,
//                    degree-5 Taylor polynomial (truncation < 4e-17);
//                    x < -707 gives 0 (subnormal results are flushed), x > 709
//                    falls back to exp().
//   log_fast(x)      x = 2^e m, m in [1,2); r = m c_j - 1 with c_j ~ 1/m from a
//                    128-entry table, |r| <= 2^-8; log1p(r) by its series to
//                    r^7 (truncation < 7e-21); falls back to log() for
//                    non-positive, subnormal, infinite or NaN x.
//   sincos_fast(p)   p = k pi/32 + r, |r| <= pi/64; sin r, cos r by their series
//                    to r^9 / r^8, then the angle-addition formulas with
//                    sin/cos(j pi/32) from a table; |p| > 1e5 falls back.
//   erfcx_poly(x)    exp(x^2) erfc(x) for 0 <= x <= 6.25: 13 pieces of width 1/2
//                    centred at k/2, degree-13 Chebyshev interpolants (relative
//                    error ~2e-16); erfcx_fast falls back to erfcx() above 6.25.
//                    (erfcx_poly_q in int_math.cuh evaluates the same pieces in
//                    fixed point on the integer pipe.)
#pragma once

#include <math.h>
#include <stdint.h>

#include "fp64_tables.cuh"

namespace ipa {

struct MathTables {
    double exp2[64];
    double linv[128];
    double ltab[128];
    double sn[64];
    double cs[64];
    double ex[fp64tab::kErfcxPieces * fp64tab::kErfcxCoeffs];
    long long exq[fp64tab::kErfcxPieces * fp64tab::kErfcxCoeffs];   // the same pieces in Q62 (int_math.cuh)
    long long sq[65], cq[65];   // sin, cos (j pi/32) in Q62 (int_math.cuh)
    long long eq[64];           // 2^(j/64) in Q62 (int_math.cuh)
};

// Block-cooperative copy of the tables into shared memory (caller syncs).
__device__ __forceinline__ void load_math_tables(MathTables* t) {
    using namespace fp64tab;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        t->exp2[i] = kExp2Tab[i];
        t->sn[i] = kSinTab[i];
        t->cs[i] = kCosTab[i];
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        t->linv[i] = kLogInv[i];
        t->ltab[i] = kLogTab[i];
    }
    for (int i = threadIdx.x; i < kErfcxPieces * kErfcxCoeffs; i += blockDim.x) {
        t->ex[i] = kErfcxTab[i];
        t->exq[i] = kErfcxQ62[i];
    }
    for (int i = threadIdx.x; i < 65; i += blockDim.x) {
        t->sq[i] = kSinQ62[i];
        t->cq[i] = kCosQ62[i];
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) t->eq[i] = kExp2Q62[i];
}

// 1.5 * 2^52: adding it rounds a double of magnitude < 2^51 to an integer held
// in the low bits of the sum's bit pattern.
constexpr double kRoundShift = 6755399441055744.0;

// Range tests on bit patterns (integer pipe; the FP64 pipe is the scarce one).
// For doubles of one sign the bit patterns are ordered like the values.
__device__ __forceinline__ bool above(double x, double c) {          // x > c, c >= 0
    return __double_as_longlong(x) > __double_as_longlong(c);
}
__device__ __forceinline__ bool below_neg(double x, double c) {      // x < c, c < 0
    return (unsigned long long)__double_as_longlong(x) > (unsigned long long)__double_as_longlong(c);
}
__device__ __forceinline__ bool abs_below(double x, double c) {      // |x| < c, c > 0
    return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) < __double_as_longlong(c);
}
__device__ __forceinline__ bool negative(double x) { return __double_as_longlong(x) < 0; }
// |x| and -x by the sign bit alone (integer pipe), so that they never take an
// FP64 instruction.
__device__ __forceinline__ double abs_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double neg_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

__device__ __forceinline__ double exp_fast(double x, const MathTables* t) {
    using namespace fp64tab;
    const double kd = fma(x, kInvLn2x64, kRoundShift);
    const int k = (int)(uint32_t)__double_as_longlong(kd);
    const double kf = kd - kRoundShift;
    double r = fma(kf, -kLn2d64Hi, x);
    r = fma(kf, -kLn2d64Lo, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    const double p = r * q;                       // e^r - 1
    const double tj = t->exp2[k & 63];
    const double v = fma(tj, p, tj);
    const long long scaled = __double_as_longlong(v) + (long long)(k >> 6) * (1ll << 52);
    if (above(x, 709.0)) return exp(x);           // overflow range: library exp
    return below_neg(x, -707.0) ? 0.0 : __longlong_as_double(scaled);
}

__device__ __forceinline__ double log_fast(double x, const MathTables* t) {
    using namespace fp64tab;
    const long long b = __double_as_longlong(x);
    // positive, normal and finite: 0x0010... <= b < 0x7FF0... (one unsigned compare)
    if ((unsigned long long)(b - 0x0010000000000000ll) >= 0x7FE0000000000000ull) return log(x);
    const int e = (int)(b >> 52) - 1023;
    const int j = (int)((b >> 45) & 127);
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    const double r = fma(m, t->linv[j], -1.0);
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(q, r, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double l = fma(r * r, q, r);            // log1p(r)
    // e as a double without a conversion instruction: 2^52 + (e + 2048) minus 2^52 + 2048
    const double ed = __longlong_as_double(0x4330000000000000ll + (long long)(e + 2048)) -
                      (4503599627370496.0 + 2048.0);
    return fma(ed, kLn2Hi, fma(ed, kLn2Lo, t->ltab[j] + l));
}

__device__ __forceinline__ void sincos_fast(double p, const MathTables* t, double* s, double* c) {
    using namespace fp64tab;
    if (!abs_below(p, 1e5)) {
        sincos(p, s, c);
        return;
    }
    const double kd = fma(p, kInvPid32, kRoundShift);
    const int k = (int)(uint32_t)__double_as_longlong(kd);
    const double kf = kd - kRoundShift;
    double r = fma(kf, -kPid32Hi, p);
    r = fma(kf, -kPid32Lo, r);
    const double r2 = r * r;
    double sp = fma(r2, 1.0 / 362880.0, -1.0 / 5040.0);
    sp = fma(sp, r2, 1.0 / 120.0);
    sp = fma(sp, r2, -1.0 / 6.0);
    const double sr = fma(sp * r2, r, r);         // sin r
    double cp = fma(r2, 1.0 / 40320.0, -1.0 / 720.0);
    cp = fma(cp, r2, 1.0 / 24.0);
    cp = fma(cp, r2, -0.5);
    const double cr = fma(cp, r2, 1.0);           // cos r
    const int j = k & 63;                          // angle j pi/32 on the circle
    const double sj = t->sn[j], cj = t->cs[j];
    *s = fma(sj, cr, cj * sr);
    *c = fma(cj, cr, -(sj * sr));
}

// 1/x to about 6e-14 relative: the FP32 reciprocal of x's leading bits
// (conversions by integer operations) refined by one FP64 Newton step, 2 FP64
// operations instead of the ~5 of a correctly rounded division.  The FP32
// seed is within 2.4e-7 of 1/x (truncation of x to 24 bits, 1 ulp of the FP32
// reciprocal), and the step squares that error.  Outside 2^-125 <= |x| <=
// 2^125 (including 0, inf, NaN) the division itself is used.
__device__ __forceinline__ double rcp_newton(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 1023 - 125 || e > 1023 + 125) return 1.0 / x;
    const unsigned xf = ((unsigned)((unsigned long long)b >> 32) & 0x80000000u) |
                        ((unsigned)(e - 1023 + 127) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu);
    const unsigned yf = __float_as_uint(__frcp_rn(__uint_as_float(xf)));
    const long long yb = ((long long)(yf & 0x80000000u) << 32) |
                         ((long long)(((yf >> 23) & 0xFFu) - 127 + 1023) << 52) | ((long long)(yf & 0x7FFFFFu) << 29);
    const double y = __longlong_as_double(yb);
    return fma(y, fma(-x, y, 1.0), y);
}

// Piecewise polynomial of erfcx on [0, 6.25]; outside, the piece index is
// clamped and the value is meaningless (callers select it away).
__device__ __forceinline__ double erfcx_poly(double x, const MathTables* t) {
    using namespace fp64tab;
    const double kd = fma(x, 2.0, kRoundShift);    // nearest piece centre k/2
    int k = (int)(uint32_t)__double_as_longlong(kd);
    k = k < 0 ? 0 : (k > kErfcxPieces - 1 ? kErfcxPieces - 1 : k);
    const double u = fma((double)k, -0.5, x);
    const double* c = t->ex + k * kErfcxCoeffs;
    double v = c[kErfcxCoeffs - 1];
#pragma unroll
    for (int i = kErfcxCoeffs - 2; i >= 0; --i) v = fma(v, u, c[i]);
    return v;
}

__device__ __forceinline__ double erfcx_fast(double x, const MathTables* t) {
    return above(x, 6.25) ? erfcx(x) : erfcx_poly(x, t);
}

}  // namespace ipa
