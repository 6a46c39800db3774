// The Faddeeva function w(z) = exp(-z^2) erfc(-i z) in the upper half plane,
// for the decay-time terms of the tagged model: the convolution of an
// oscillating exponential e^{-(Gamma - i Dm) t} with a Gaussian is a complex
// erfc, which Sec. 2 and the symbolic-programming section of the paper
// evaluate through w(z).
//
// Method: Weideman's rational approximation (J.A.C. Weideman, "Computation of
// the complex error function", SIAM J. Numer. Anal. 31 (1994) 1497).  For
// Im z > 0, w(z) = (i/pi) int e^{-t^2} / (z - t) dt.  With t = L tan(theta/2),
// e^{-t^2} (L^2 + t^2) = sum_n a_n e^{i n theta} (even in theta) and
// e^{i theta} = (L + i t) / (L - i t); integrating each term by residues
// (closing the contour above for n >= 0, below for n < 0) gives
//   w(z) = 1 / (sqrt(pi) (L - i z)) + 2 sum_{n>=1} a_n Z^{n-1} / (L - i z)^2,
//   Z = (L + i z) / (L - i z),
// truncated at n = N = 40 with L = 2^(-1/4) sqrt(N).  The coefficients are
// generated in 60-digit arithmetic (gen_fp64_tables.py).  Measured against
// mpmath over 0 <= Re z <= 8, 0 <= Im z <= 1000 the relative error is below
// 7e-16 in FP64 (by the symmetry w(-conj z) = conj w(z) the same holds for
// Re z < 0).  |Z| <= 1 in the closed upper half plane, so Horner's rule is
// stable; |L - i z| >= L keeps every division away from zero.
//
// The 39 complex Horner steps (four products each, 156 FP64 operations) run
// on the integer pipe: Z in Q62, the partial sums p in Q59 (|p| <= sum |a_n|
// = 12.64 < 16, so no step overflows), each product the high half of a
// 64 x 64 -> 128-bit product.  A floored high half is half a unit low on
// average; the imaginary part adds two such products per step and gets one
// unit back, the real part subtracts them and needs none.  The error of p is
// a few 2^-57 (1e-17 absolute against |p| of order 1), and it reaches w
// divided by |L - i z|^2 >= L^2.  Only the division, Z and the final
// combination are FP64.
#pragma once

#include <math.h>

#include "fp64_tables.cuh"
#include "int_math.cuh"

namespace ipa {

// w(x + i y) for y >= 0: about 20 FP64 operations, one division and the
// fixed-point Horner sum.  It is evaluated at |x| and conjugated for x < 0
// (w(-conj z) = conj w(z)), so that symmetry holds bit for bit although the
// floored products are not odd.  The Horner loop is not unrolled (unrolled, it
// overflowed the instruction cache of the tagged kernel).
__device__ __forceinline__ void faddeeva_uhp(double xs, double y, double* wr, double* wi) {
    using namespace fp64tab;
    const double x = abs_bits(xs);
    // d = L - i z = (L + y) - i x;  1/d = ((L + y) + i x) / |d|^2
    const double dr = kWeidL + y;
    const double inv = 1.0 / fma(dr, dr, x * x);
    const double er = dr * inv, ei = x * inv;
    // Z = (L + i z) / d = ((L - y) + i x) / d
    const double nr = kWeidL - y;
    const double Zr = fma(nr, er, -(x * ei)), Zi = fma(nr, ei, x * er);
    const long long zr = to_q62_nb(Zr), zi = to_q62_nb(Zi);     // |Z| <= 1 (+ rounding)
    long long qr = kWeidAQ59[kWeidN - 1], qi = 0;
#pragma unroll 1
    for (int k = kWeidN - 2; k >= 0; --k) {
        const long long t = kWeidAQ59[k] + (long long)((unsigned long long)(__mul64hi(qr, zr) - __mul64hi(qi, zi)) << 2);
        qi = (long long)((unsigned long long)(__mul64hi(qr, zi) + __mul64hi(qi, zr) + 1) << 2);
        qr = t;
    }
    const double pr = q62_to_double_nb(qr, 3), pi = q62_to_double_nb(qi, 3);
    // w = (2 p / d + 1/sqrt(pi)) / d
    const double tr = fma(2.0, fma(pr, er, -(pi * ei)), kInvSqrtPi);
    const double ti = 2.0 * fma(pr, ei, pi * er);
    *wr = fma(tr, er, -(ti * ei));
    const double wim = fma(tr, ei, ti * er);
    *wi = negative(xs) ? neg_bits(wim) : wim;
}

// w(z) anywhere: the upper half plane directly, the lower by the reflection
// w(z) = 2 exp(-z^2) - w(-z) (library exp and sincos; it overflows where
// exp(-z^2) does).
__device__ __forceinline__ void faddeeva(double x, double y, double* wr, double* wi) {
    if (!(y < 0.0)) {
        faddeeva_uhp(x, y, wr, wi);
        return;
    }
    double ur, ui;
    faddeeva_uhp(-x, -y, &ur, &ui);
    // exp(-z^2) = exp(y^2 - x^2) (cos(2xy) - i sin(2xy))
    const double m = 2.0 * exp((y - x) * (y + x));
    double s, c;
    sincos(2.0 * x * y, &s, &c);
    *wr = fma(m, c, -ur);
    *wi = fma(-m, s, -ui);
}

}  // namespace ipa
