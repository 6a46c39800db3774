// FP64 sin/cos and exp computed on the integer pipe.
//
// On this GPU the FP64 pipe issues 2 operations per clock per SM and is what
// bounds the likelihood kernel, while the integer pipe issues 64.  These
// functions take a double, do the range reduction and the polynomial in
// 64-bit fixed point (64 x 64 -> 128-bit products on the integer pipe, no
// FP64 instruction) and round the fixed-point result once to a double:
//
//   sincos_int  |phi| < 4 (sincos_int_wide: |phi| < 1024, for phases): phi in
//               Q61 (Q53), k = nearest multiple of pi/32,
//               r = phi - k pi/32 in Q64 (|r| <= pi/64), Taylor polynomials of
//               sin r to r^9 and cos r to r^8 (truncation below 1e-19), then
//               sin phi = S_k cos r + C_k sin r, cos phi = C_k cos r - S_k sin r
//               with S_k, C_k = sin, cos (k pi/32) in Q62.  Absolute error
//               before the final rounding: a few 2^-62 (the angular functions
//               need absolute, not relative, accuracy).
//   exp_int     -705 < a < 709: |a| in Q53 (exact for |a| >= 1/2, within
//               2^-53 otherwise), k = nearest integer to a 64/ln2,
//               r = a - k ln2/64 in Q64 with ln2/64 to 128 bits (|r| <=
//               ln2/128), e^r - 1 to r^6 (truncation below 3e-20), times
//               2^(j/64) (Q62, j = k mod 64) and 2^floor(k/64).  Relative error
//               before the final rounding: about 2^-53 from the input
//               quantisation for |a| < 1/2, a few 2^-62 otherwise.
//   erfcx_poly_q  0 <= x <= 6.25: x in Q60, k = nearest multiple of 1/2 (piece
//               centre), u = x - k/2 in Q63 (|u| <= 1/4), the degree-13
//               Chebyshev interpolant of the piece (monomials in u, Q62) by
//               Horner's rule with 64 x 64 -> 128-bit products.  Absolute error
//               before the final rounding below 2^-61 (the values are above
//               0.088, so below 2e-17 relative, plus the interpolant's own
//               ~1e-16).
//
// Outside these ranges sincos_int and exp_int fall back to the table-driven
// FP64 functions; erfcx_fast_q falls back to the library erfcx.
#pragma once

#include "fp64_math.cuh"

namespace ipa {

// Signed Q62 value v to the nearest double, times 2^e2 (|v| < 2^63; the result
// must be a normal double).
__device__ __forceinline__ double q62_to_double(long long v, int e2) {
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    a <<= lz;                                               // leading one at bit 63
    unsigned long long m = a >> 11;                         // 53 bits
    const unsigned long long rem = a & 0x7FFull;
    m += (rem > 0x400ull) || (rem == 0x400ull && (m & 1ull));   // nearest, ties to even
    // value = m 2^(1 - lz - 52 + e2); m includes the hidden bit, which adds one to
    // the exponent field (and a rounding carry to 2^53 adds another)
    const long long field = (long long)(1 - lz + e2 + 1022);
    return __longlong_as_double((long long)(sign | (((unsigned long long)field << 52) + m)));
}

// sin(k pi/32 +- r) and cos(k pi/32 +- r) in Q62 from k (0..64) and |r| in
// Q64 (|r| <= pi/64; rneg: the sign of r): Taylor polynomials of sin r and
// 1 - cos r, then the angle-addition formulas with S_k, C_k from the tables.
__device__ __forceinline__ void sincos_poly_q62(int k, unsigned long long r, bool rneg, const MathTables* t,
                                                long long* sv, long long* cv) {
    using namespace fp64tab;
    const unsigned long long z = __umul64hi(r, r);                     // r^2
    unsigned long long p = kSinC9Q64;
    p = kSinC7Q64 - __umul64hi(z, p);
    p = kSinC5Q64 - __umul64hi(z, p);
    p = kSinC3Q64 - __umul64hi(z, p);
    const long long sr = (long long)(r - __umul64hi(r, __umul64hi(z, p)));   // |sin r| in Q64, < 2^60
    unsigned long long q = kCosC8Q64;
    q = kCosC6Q64 - __umul64hi(z, q);
    q = kCosC4Q64 - __umul64hi(z, q);
    q = kCosC2Q64 - __umul64hi(z, q);
    const long long cm = (long long)__umul64hi(z, q);                  // 1 - cos r in Q64, < 2^54
    const long long srs = rneg ? -sr : sr;
    const long long Sk = t->sq[k], Ck = t->cq[k];                      // Q62
    // S_k (1 - cm) + C_k sin r and C_k (1 - cm) - S_k sin r, in Q62
    *sv = Sk - __mul64hi(Sk, cm) + __mul64hi(Ck, srs);
    *cv = Ck - __mul64hi(Ck, cm) - __mul64hi(Sk, srs);
}

// sin and cos of |phi| in signed Q62 (|phi| < 4, the caller checks), before
// the sign of phi is applied to the sine.
__device__ __forceinline__ void sincos_q62(unsigned long long b, const MathTables* t, long long* sv,
                                           long long* cv) {
    using namespace fp64tab;
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = E + 9;                                   // |phi| in Q61
    const unsigned long long X = sh >= 0 ? M << sh : (sh > -64 ? M >> -sh : 0ull);
    const unsigned long long U = __umul64hi(X, kTwoOverPiQ64);        // |phi| 32/pi in Q57
    const unsigned long long k = (U + (1ull << 56)) >> 57;
    const long long rq = (long long)(U - (k << 57));                   // |rq| <= 2^56
    const bool rneg = rq < 0;
    const unsigned long long ra = rneg ? (unsigned long long)(-rq) : (unsigned long long)rq;
    const unsigned long long r = __umul64hi(ra << 7, kPiOver32Q64);   // |r| in Q64
    sincos_poly_q62((int)k, r, rneg, t, sv, cv);
}

// sin and cos of phi for |phi| < 4 (else the table-driven sincos_fast).
__device__ __forceinline__ void sincos_int(double phi, const MathTables* t, double* s, double* c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(phi);
    if ((int)((b >> 52) & 0x7FFull) - 1023 > 1) {           // |phi| >= 4, inf, NaN
        sincos_fast(phi, t, s, c);
        return;
    }
    long long sv, cv;
    sincos_q62(b, t, &sv, &cv);
    const double sd = q62_to_double(sv, 0);
    *s = (b >> 63) ? -sd : sd;
    *c = q62_to_double(cv, 0);
}

// sin and cos of phi for |phi| < 1024 (else the table-driven sincos_fast), for
// phases such as Dm t: |phi| in Q53 (exact for |phi| >= 1/2, within 2^-53
// otherwise), k = nearest integer to |phi| 32/pi, r = |phi| - k pi/32 in Q64
// with pi/32 to 128 bits (error below 2^-110), then the polynomials of
// sincos_poly_q62 with the table entry k mod 64.
__device__ __forceinline__ void sincos_int_wide(double phi, const MathTables* t, double* s, double* c) {
    using namespace fp64tab;
    const unsigned long long b = (unsigned long long)__double_as_longlong(phi);
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    if (E > 9) {                                            // |phi| >= 1024, inf, NaN
        sincos_fast(phi, t, s, c);
        return;
    }
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = E + 1;                                   // |phi| in Q53
    const unsigned long long A = sh >= 0 ? M << sh : (sh > -64 ? M >> -sh : 0ull);
    // k = round(|phi| 32/pi): A (Q53) x 32/pi (Q59) >> 64 is Q48
    const unsigned long long P = __umul64hi(A, k32OverPiQ59);
    const unsigned long long k = (P + (1ull << 47)) >> 48;
    const unsigned __int128 kl = (unsigned __int128)k * kPiOver32Q128Hi +
                                 (((unsigned __int128)k * kPiOver32Q128Lo) >> 64);
    const long long r = (long long)(((__int128)A << 11) - (__int128)kl);    // Q64, |r| <= pi/64
    const bool rneg = r < 0;
    long long sv, cv;
    sincos_poly_q62((int)(k & 63ull), rneg ? (unsigned long long)(-r) : (unsigned long long)r, rneg, t, &sv, &cv);
    const double sd = q62_to_double(sv, 0);
    *s = (b >> 63) ? -sd : sd;
    *c = q62_to_double(cv, 0);
}

// e^a for -705 < a < 709 (else the table-driven exp_fast).
__device__ __forceinline__ double exp_int(double a, const MathTables* t) {
    using namespace fp64tab;
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    const bool neg = (b >> 63) != 0;
    if (E > 9 || (neg ? below_neg(a, -705.0) : above(a, 709.0))) return exp_fast(a, t);
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = E + 1;                                   // |a| in Q53
    const unsigned long long A = sh >= 0 ? M << sh : (sh > -64 ? M >> -sh : 0ull);
    // k = round(|a| 64/ln2): A (Q53) x 64/ln2 (Q56) >> 64 is Q45
    const unsigned long long P = __umul64hi(A, kInvLn2x64Q56);
    const unsigned long long k = (P + (1ull << 44)) >> 45;
    // r = |a| - k ln2/64 in Q64, from A << 11 minus k times ln2/64 to 128 bits
    const unsigned __int128 kl = (unsigned __int128)k * kLn2d64Q128Hi +
                                 (((unsigned __int128)k * kLn2d64Q128Lo) >> 64);
    const long long r = (long long)(((__int128)A << 11) - (__int128)kl);
    const long long rs = neg ? -r : r;
    const long long ks = neg ? -(long long)k : (long long)k;
    // e^rs - 1 = rs + rs^2 (1/2 + rs (1/6 + rs (1/24 + rs (1/120 + rs/720))))  (Q63 inner)
    long long v = kExpC6Q63;
    v = kExpC5Q63 + __mul64hi(rs, v);
    v = kExpC4Q63 + __mul64hi(rs, v);
    v = kExpC3Q63 + __mul64hi(rs, v);
    v = kExpC2Q63 + __mul64hi(rs, v);
    const long long pm = rs + (__mul64hi(__mul64hi(rs, v), rs) << 1);   // Q64
    const long long T = t->eq[ks & 63];                                  // 2^(j/64) in Q62
    const long long y = T + __mul64hi(T, pm);                            // Q62
    return q62_to_double(y, (int)(ks >> 6));
}

// x in signed Q62 for |x| <= 1 (the caller checks): exact when |x| >= 2^-10,
// truncated to 2^-62 below.
__device__ __forceinline__ long long to_q62(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int sh = (int)((b >> 52) & 0x7FFull) - 1023 + 10;
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const long long v = (long long)(sh >= 0 ? M << sh : (sh > -64 ? M >> -sh : 0ull));
    return (b >> 63) ? -v : v;
}

// (a b) in Q62 for a, b in signed Q62 with |a b| < 2: the high product shifted
// left by 2 (the two lowest bits are lost: error below 2^-60).
__device__ __forceinline__ long long mul_q62(long long a, long long b) { return __mul64hi(a, b) << 2; }

constexpr long long kOneQ62 = 1ll << 62;

// sqrt(x) in Q62 for x in [0, 1] given in Q124 (a product of two Q62 values,
// so that small x keep their relative precision): an FP32 seed refined by two
// Newton steps on the exact 128-bit residual (relative error about 2^-60, plus
// 2^-62 absolute from the final shift).
__device__ __forceinline__ long long sqrt_q124(unsigned __int128 X) {
    if (X == 0) return 0;
    const unsigned long long xh = (unsigned long long)(X >> 64), xl = (unsigned long long)X;
    const int lz = xh ? __clzll((long long)xh) : 64 + __clzll((long long)xl);
    const int d = 124 - (127 - lz);                    // >= 0: x <= 1
    const int s = d & ~1;                              // even shift: xn = Xn 2^-124 in [1/2, 2)
    const unsigned __int128 Xn = X << s;
    const int top = 127 - lz + s;                      // 123 or 124
    const unsigned fb = ((unsigned)(top - 124 + 127) << 23) | ((unsigned)(Xn >> (top - 23)) & 0x7FFFFFu);
    const float y0f = rsqrtf(__uint_as_float(fb));     // ~1/sqrt(xn) in (0.7, 1.42)
    const unsigned yb = __float_as_uint(y0f);
    const int ye = (int)((yb >> 23) & 0xFF) - 127;     // -1 or 0
    const long long Y0 = (long long)(((unsigned long long)((yb & 0x7FFFFF) | 0x800000)) << (39 + ye));
    long long Q = mul_q62((long long)(Xn >> 62), Y0);  // ~sqrt(xn) in Q62
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const __int128 R = (__int128)Xn - (__int128)Q * Q;               // residual in Q124
        Q += __mul64hi((long long)(R >> 62), Y0) << 1;                    // + R y0 / 2
    }
    return Q >> (s >> 1);
}

// 1 - x^2 in Q62 for x in signed Q62, |x| <= 1, from the exact square
// (error below 2^-62).
__device__ __forceinline__ long long one_minus_sq_q62(long long x) {
    return (long long)((((unsigned __int128)1 << 124) - (unsigned __int128)((__int128)x * x)) >> 62);
}

// Whether basis_q62 keeps its accuracy for these angles: |phi| < 4 and
// |cos thK|, |cos thmu| < 1 - 2^-17, so that sin^2 = 1 - cos^2 >= 2^-16 and its
// fixed-point error (2^-60 absolute) stays below 2^-44 relative.  Outside (about
// 1.5e-5 of uniformly distributed angles, and invalid |cos| > 1 or NaN) the
// caller uses the FP64 basis.
__device__ __forceinline__ bool basis_q62_ok(double ck, double cl, double phi) {
    constexpr double kMaxCos = 1.0 - 0x1p-17;
    return abs_below(ck, kMaxCos) && abs_below(cl, kMaxCos) && abs_below(phi, 4.0);
}

// The ten unscaled angular products f'_k (sec. 4 helicity basis, without their
// constant factors) in signed Q62 (absolute error a few 2^-60), for angles
// that pass basis_q62_ok.  sin thK sin thmu = sqrt((1 - cos^2 thK)(1 - cos^2 thmu)).
__device__ __forceinline__ void basis_q62(double ck, double cl, double phi, const MathTables* t, long long F[10]) {
    const unsigned long long pb = (unsigned long long)__double_as_longlong(phi);
    long long sp, cp;
    sincos_q62(pb, t, &sp, &cp);
    if (pb >> 63) sp = -sp;
    const long long CK = to_q62(ck), CL = to_q62(cl);
    const long long sk2 = one_minus_sq_q62(CK), sl2 = one_minus_sq_q62(CL);
    const long long ck2 = kOneQ62 - sk2, cl2 = kOneQ62 - sl2;
    const long long cp2 = mul_q62(cp, cp);
    const unsigned __int128 sksl2_124 = (unsigned __int128)((__int128)sk2 * sl2);
    const long long sksl2 = (long long)(sksl2_124 >> 62);
    const long long q = sqrt_q124(sksl2_124);
    const long long slcp2 = mul_q62(sl2, cp2);
    F[0] = mul_q62(ck2, sl2);
    F[1] = mul_q62(sk2, kOneQ62 - slcp2);
    F[2] = mul_q62(sk2, slcp2 + cl2);
    F[3] = mul_q62(sksl2, mul_q62(sp, cp));
    const long long a = mul_q62(q, mul_q62(CK, CL));
    F[4] = mul_q62(a, cp);
    F[5] = mul_q62(a, sp);
    F[6] = sl2;
    const long long bq = mul_q62(q, CL);
    F[7] = mul_q62(bq, cp);
    F[8] = mul_q62(bq, sp);
    F[9] = mul_q62(CK, sl2);
}

// ---- branch-free forms for software-pipelined event loops ----
// The functions below return the same values as the ones above for inputs in
// their ranges (exp_int_ok, basis_q62_ok), without a branch, so that a warp can
// evaluate them for the next event in one basic block together with the FP64
// work of the current event (the GPU overlaps FP64 and integer instructions of
// one warp, not of different warps) and fix up the rare lanes outside the
// ranges afterwards.  Outside the ranges the values are unspecified; every
// shift stays below 64 and every table index inside its table.

// q62_to_double, also for v = 0 (which gives +0).
__device__ __forceinline__ double q62_to_double_nb(long long v, int e2) {
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);                   // 64 for a = 0
    a <<= (lz & 63);
    unsigned long long m = a >> 11;
    const unsigned long long rem = a & 0x7FFull;
    m += (rem > 0x400ull) || (rem == 0x400ull && (m & 1ull));
    const long long field = (long long)(1 - lz + e2 + 1022);
    const long long bits = (long long)(sign | (((unsigned long long)field << 52) + m));
    return __longlong_as_double(v == 0 ? 0ll : bits);
}

// M 2^sh for a 53-bit M and any sh (0 for sh <= -64; sh >= 64 wraps, for
// inputs outside the ranges only).
__device__ __forceinline__ unsigned long long shift_nb(unsigned long long M, int sh) {
    const unsigned long long up = M << (sh & 63);
    const unsigned long long dn = M >> ((-sh) & 63);
    return sh >= 0 ? up : (sh > -64 ? dn : 0ull);
}

// Range of exp_int's fixed-point path: -705 < a < 709.
__device__ __forceinline__ bool exp_int_ok(double a) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    return !(E > 9 || ((b >> 63) ? below_neg(a, -705.0) : above(a, 709.0)));
}

// exp_int without its range test (the caller checks exp_int_ok).
__device__ __forceinline__ double exp_int_nb(double a, const MathTables* t) {
    using namespace fp64tab;
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    const bool neg = (b >> 63) != 0;
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned long long A = shift_nb(M, E + 1);       // |a| in Q53
    const unsigned long long P = __umul64hi(A, kInvLn2x64Q56);
    const unsigned long long k = (P + (1ull << 44)) >> 45;
    const unsigned __int128 kl = (unsigned __int128)k * kLn2d64Q128Hi +
                                 (((unsigned __int128)k * kLn2d64Q128Lo) >> 64);
    const long long r = (long long)(((__int128)A << 11) - (__int128)kl);
    const long long rs = neg ? -r : r;
    const long long ks = neg ? -(long long)k : (long long)k;
    long long v = kExpC6Q63;
    v = kExpC5Q63 + __mul64hi(rs, v);
    v = kExpC4Q63 + __mul64hi(rs, v);
    v = kExpC3Q63 + __mul64hi(rs, v);
    v = kExpC2Q63 + __mul64hi(rs, v);
    const long long pm = rs + (__mul64hi(__mul64hi(rs, v), rs) << 1);
    const long long T = t->eq[ks & 63];
    const long long y = T + __mul64hi(T, pm);
    return q62_to_double_nb(y, (int)(ks >> 6));
}

// sincos_q62 for any bit pattern (the table index clamped to the table).
__device__ __forceinline__ void sincos_q62_nb(unsigned long long b, const MathTables* t, long long* sv,
                                              long long* cv) {
    using namespace fp64tab;
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned long long X = shift_nb(M, E + 9);       // |phi| in Q61
    const unsigned long long U = __umul64hi(X, kTwoOverPiQ64);
    const unsigned long long k = (U + (1ull << 56)) >> 57;
    const long long rq = (long long)(U - (k << 57));
    const bool rneg = rq < 0;
    const unsigned long long ra = rneg ? (unsigned long long)(-rq) : (unsigned long long)rq;
    const unsigned long long r = __umul64hi(ra << 7, kPiOver32Q64);
    sincos_poly_q62(k > 64ull ? 64 : (int)k, r, rneg, t, sv, cv);
}

// to_q62 for any double (unspecified outside |x| <= 1).
__device__ __forceinline__ long long to_q62_nb(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const long long v = (long long)shift_nb(M, (int)((b >> 52) & 0x7FFull) - 1023 + 10);
    return (b >> 63) ? -v : v;
}

// sqrt_q124 without the branch on zero.
__device__ __forceinline__ long long sqrt_q124_nb(unsigned __int128 X) {
    const bool zero = X == 0;
    const unsigned __int128 Xs = zero ? (unsigned __int128)1 : X;
    const unsigned long long xh = (unsigned long long)(Xs >> 64), xl = (unsigned long long)Xs;
    const int lz = xh ? __clzll((long long)xh) : 64 + __clzll((long long)xl);
    const int d = 124 - (127 - lz);
    const int s = d & ~1;
    const unsigned __int128 Xn = Xs << (s & 127);
    const int top = 127 - lz + s;
    const unsigned fb = ((unsigned)(top - 124 + 127) << 23) | ((unsigned)(Xn >> ((top - 23) & 127)) & 0x7FFFFFu);
    const float y0f = rsqrtf(__uint_as_float(fb));
    const unsigned yb = __float_as_uint(y0f);
    const int ye = (int)((yb >> 23) & 0xFF) - 127;
    const long long Y0 = (long long)(((unsigned long long)((yb & 0x7FFFFF) | 0x800000)) << ((39 + ye) & 63));
    long long Q = mul_q62((long long)(Xn >> 62), Y0);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const __int128 R = (__int128)Xn - (__int128)Q * Q;
        Q += __mul64hi((long long)(R >> 62), Y0) << 1;
    }
    return zero ? 0 : Q >> ((s >> 1) & 63);
}

// basis_q62 without branches (the caller checks basis_q62_ok).
__device__ __forceinline__ void basis_q62_nb(double ck, double cl, double phi, const MathTables* t,
                                             long long F[10]) {
    const unsigned long long pb = (unsigned long long)__double_as_longlong(phi);
    long long sp, cp;
    sincos_q62_nb(pb, t, &sp, &cp);
    sp = (pb >> 63) ? -sp : sp;
    const long long CK = to_q62_nb(ck), CL = to_q62_nb(cl);
    const long long sk2 = one_minus_sq_q62(CK), sl2 = one_minus_sq_q62(CL);
    const long long ck2 = kOneQ62 - sk2, cl2 = kOneQ62 - sl2;
    const long long cp2 = mul_q62(cp, cp);
    const unsigned __int128 sksl2_124 = (unsigned __int128)((__int128)sk2 * sl2);
    const long long sksl2 = (long long)(sksl2_124 >> 62);
    const long long q = sqrt_q124_nb(sksl2_124);
    const long long slcp2 = mul_q62(sl2, cp2);
    F[0] = mul_q62(ck2, sl2);
    F[1] = mul_q62(sk2, kOneQ62 - slcp2);
    F[2] = mul_q62(sk2, slcp2 + cl2);
    F[3] = mul_q62(sksl2, mul_q62(sp, cp));
    const long long a = mul_q62(q, mul_q62(CK, CL));
    F[4] = mul_q62(a, cp);
    F[5] = mul_q62(a, sp);
    F[6] = sl2;
    const long long bq = mul_q62(q, CL);
    F[7] = mul_q62(bq, cp);
    F[8] = mul_q62(bq, sp);
    F[9] = mul_q62(CK, sl2);
}

// erfcx(x) = exp(x^2) erfc(x) for 0 <= x <= 6.25 from the piecewise
// polynomial of fp64_tables.cuh (erfcx_poly's pieces), on the integer pipe.  x
// above 6.25, infinite or NaN is evaluated as 6.25 and a negative x as |x|: the
// value is then meaningless and callers select it away (erfcx_fast_q).  The
// Horner loop is not unrolled: unrolled, the 64-bit products of the kernels
// that call this twice per event overflowed the instruction cache.
__device__ __forceinline__ double erfcx_poly_q(double x, const MathTables* t) {
    using namespace fp64tab;
    long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll;
    b = b > 0x4019000000000000ll ? 0x4019000000000000ll : b;      // 6.25
    const unsigned long long M = ((unsigned long long)b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned long long X = shift_nb(M, (int)(b >> 52) - 1023 + 8);   // x in Q60, < 2^63
    int k = (int)((X + (1ull << 58)) >> 59);                      // nearest piece centre k/2
    k = k > kErfcxPieces - 1 ? kErfcxPieces - 1 : k;
    const long long u = (long long)((X - ((unsigned long long)k << 59)) << 3);   // Q63, |u| <= 2^61
    const long long* c = t->exq + k * kErfcxCoeffs;
    long long v = c[kErfcxCoeffs - 1];
#pragma unroll 1
    for (int i = kErfcxCoeffs - 2; i >= 0; --i)
        v = c[i] + (long long)((unsigned long long)__mul64hi(v, u) << 1);   // |v| < 1.5 in Q62
    return q62_to_double_nb(v, 0);
}

__device__ __forceinline__ double erfcx_fast_q(double x, const MathTables* t) {
    return above(x, 6.25) ? erfcx(x) : erfcx_poly_q(x, t);
}

}  // namespace ipa
