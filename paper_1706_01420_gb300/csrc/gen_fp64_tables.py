"""Generate fp64_tables.cuh: the tables and split constants of the library's
FP64 elementary functions (fp64_math.cuh), computed in 60-digit arithmetic
with mpmath and rounded once to double.

  exp:    T_j = 2^(j/64), j = 0..63; 64/ln2; ln2/64 as hi + lo
  log:    c_j = 1/(1 + (j + 1/2)/128) rounded to double, j = 0..127, and
          L_j = -log(c_j) of that rounded c_j (so log m = L_j + log1p(m c_j - 1)
          holds exactly); ln2
  sincos: S_j = sin(j pi/32), C_j = cos(j pi/32), j = 0..63; 32/pi; pi/32 as hi + lo
  erfcx:  erfcx(x) = exp(x^2) erfc(x) on x in [0, 6.25] as 13 pieces centred at
          k/2 (k = 0..12), each the degree-13 Chebyshev interpolant on
          [k/2 - 0.26, k/2 + 0.26] written as monomials in u = x - k/2, each
          coefficient rounded once to double and once to signed Q62 (for the
          fixed-point evaluation: every coefficient and every partial Horner
          sum over |u| <= 1/4 is below 1.5 in magnitude, checked here);

the coefficients of the Faddeeva function (faddeeva.cuh), Weideman's rational
approximation (SIAM J. Numer. Anal. 31 (1994) 1497) with N = 40 and
L = 2^(-1/4) sqrt(N):

  a_n = (1/pi) int_0^pi psi(theta) cos(n theta) dtheta,  n = 1..N,
  psi = exp(-t^2) (L^2 + t^2) at t = L tan(theta / 2),

by the midpoint rule with 1024 nodes (psi is smooth and periodic, so the rule
converges geometrically; 512 nodes give the same doubles), each rounded once
to signed Q59 (the Horner sum in Z, |Z| <= 1, is evaluated in fixed point and
never exceeds sum |a_n| = 12.64 < 16, checked here), and
the fixed-point tables and constants of the integer-pipe functions
(int_math.cuh), each the exact value rounded once to an integer:

  sincos: round(sin(j pi/32) 2^62), round(cos(j pi/32) 2^62), j = 0..64;
          2/pi and pi/32 in Q64; 32/pi in Q59 and pi/32 in Q128 as two
          64-bit words (the wide-range reduction); the Taylor coefficients 1/3!, .., 1/9! of sin
          and 1/2!, .., 1/8! of cos in Q64
  exp:    round(2^(j/64) 2^62), j = 0..63; 64/ln2 in Q56; ln2/64 in Q128 as
          two 64-bit words; 1/2!, .., 1/6! in Q63

Run: python paper_1706_01420_gb300/csrc/gen_fp64_tables.py  (rewrites the header)
"""
from __future__ import annotations

import os

import mpmath as mp

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))

ERFCX_PIECES = 13
ERFCX_DEG = 13
ERFCX_HALF = mp.mpf("0.26")


def d(x) -> float:
    return float(mp.mpf(x))


def split(x):
    hi = d(x)
    lo = d(mp.mpf(x) - mp.mpf(hi))
    return hi, lo


def cheb_monomial(f, a, b, n):
    c = (a + b) / 2
    h = (b - a) / 2
    nodes = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (n + 1)) for k in range(n + 1)]
    vals = [f(c + h * t) for t in nodes]
    ck = []
    for j in range(n + 1):
        s = mp.fsum(vals[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / (n + 1)) for k in range(n + 1))
        ck.append(2 * s / (n + 1) if j else s / (n + 1))
    T = [[mp.mpf(0)] * (n + 1) for _ in range(n + 1)]
    T[0][0] = mp.mpf(1)
    T[1][1] = mp.mpf(1)
    for j in range(2, n + 1):
        for i in range(n + 1):
            T[j][i] = (2 * T[j - 1][i - 1] if i else 0) - T[j - 2][i]
    mono_t = [mp.fsum(ck[j] * T[j][i] for j in range(n + 1)) for i in range(n + 1)]
    return [mono_t[i] / h ** i for i in range(n + 1)]


def erfcx(x):
    return mp.exp(x * x) * mp.erfc(x)


def q(x, bits: int) -> int:
    """round(x 2^bits) as a Python integer."""
    return int(mp.nint(mp.mpf(x) * mp.power(2, bits)))


def fmt_int(vals, per_line=3, suffix="ll"):
    out = []
    for i in range(0, len(vals), per_line):
        out.append("    " + ", ".join(f"{v}{suffix}" for v in vals[i:i + per_line]) + ",")
    return "\n".join(out)


def fmt(vals, per_line=3):
    out = []
    for i in range(0, len(vals), per_line):
        out.append("    " + ", ".join(repr(v) for v in vals[i:i + per_line]) + ",")
    return "\n".join(out)


WEID_N = 40
WEID_NODES = 1024


def weideman(n_terms: int, nodes: int):
    """L and the Fourier cosine coefficients a_1..a_N of psi (see the docstring)."""
    L = mp.power(2, mp.mpf(-1) / 4) * mp.sqrt(n_terms)
    th = [mp.pi * (k + mp.mpf(1) / 2) / nodes for k in range(nodes)]
    psi = []
    for t in th:
        x = L * mp.tan(t / 2)
        psi.append(mp.exp(-x * x) * (L * L + x * x))
    # (1/pi) * (pi / nodes) * sum: the midpoint rule on (0, pi)
    a = [mp.fsum(psi[k] * mp.cos(n * th[k]) for k in range(nodes)) / nodes for n in range(1, n_terms + 1)]
    return L, a


def main():
    exp_tab = [d(mp.power(2, mp.mpf(j) / 64)) for j in range(64)]
    ln2 = mp.log(2)
    inv_ln2_64 = d(64 / ln2)
    ln2_64_hi, ln2_64_lo = split(ln2 / 64)
    log_c = [d(1 / (1 + (mp.mpf(j) + mp.mpf(1) / 2) / 128)) for j in range(128)]
    log_l = [d(-mp.log(mp.mpf(c))) for c in log_c]
    sin_tab = [d(mp.sin(j * mp.pi / 32)) for j in range(64)]
    cos_tab = [d(mp.cos(j * mp.pi / 32)) for j in range(64)]
    inv_pi_32 = d(32 / mp.pi)
    pi_32_hi, pi_32_lo = split(mp.pi / 32)
    sin_q62 = [q(mp.sin(j * mp.pi / 32), 62) for j in range(65)]
    cos_q62 = [q(mp.cos(j * mp.pi / 32), 62) for j in range(65)]
    exp2_q62 = [q(mp.power(2, mp.mpf(j) / 64), 62) for j in range(64)]
    ln2_64_q128 = q(ln2 / 64, 128)
    fact = [mp.factorial(n) for n in range(10)]
    erfcx_tab, erfcx_q62 = [], []
    for k in range(ERFCX_PIECES):
        c = mp.mpf(k) / 2
        coef = cheb_monomial(erfcx, c - ERFCX_HALF, c + ERFCX_HALF, ERFCX_DEG)
        # partial Horner sums on a grid of |u| <= 1/4 (the sums are polynomials
        # of low degree in u with decaying coefficients: the grid maximum is the
        # maximum to well within the margin to 2)
        worst = max(abs(v) for v in coef)
        for i in range(201):
            u = mp.mpf(i) / 400 - mp.mpf(1) / 4
            v = coef[-1]
            for j in range(len(coef) - 2, -1, -1):
                v = coef[j] + v * u
                worst = max(worst, abs(v))
        assert worst < 1.5, (k, worst)
        erfcx_tab.extend(d(v) for v in coef)
        erfcx_q62.extend(q(v, 62) for v in coef)

    weid_L, weid_a = weideman(WEID_N, WEID_NODES)
    assert mp.fsum(abs(v) for v in weid_a) < 13
    weid_q59 = [q(v, 59) for v in weid_a]

    text = f"""// Generated by gen_fp64_tables.py (mpmath, 60 digits, rounded once to double
// or to an integer).
// Do not edit by hand.
#pragma once

namespace ipa {{
namespace fp64tab {{

constexpr double kInvLn2x64 = {inv_ln2_64!r};      // 64 / ln 2
constexpr double kLn2d64Hi = {ln2_64_hi!r};        // ln 2 / 64, high part
constexpr double kLn2d64Lo = {ln2_64_lo!r};        // ln 2 / 64, low part
constexpr double kLn2Hi = {split(ln2)[0]!r};        // ln 2, high part
constexpr double kLn2Lo = {split(ln2)[1]!r};        // ln 2, low part
constexpr double kInvPid32 = {inv_pi_32!r};        // 32 / pi
constexpr double kPid32Hi = {pi_32_hi!r};          // pi / 32, high part
constexpr double kPid32Lo = {pi_32_lo!r};          // pi / 32, low part
constexpr int kErfcxPieces = {ERFCX_PIECES};
constexpr int kErfcxCoeffs = {ERFCX_DEG + 1};

// 2^(j/64)
__device__ const double kExp2Tab[64] = {{
{fmt(exp_tab)}
}};

// c_j ~ 1/(1 + (j + 1/2)/128) and L_j = -log(c_j)
__device__ const double kLogInv[128] = {{
{fmt(log_c)}
}};
__device__ const double kLogTab[128] = {{
{fmt(log_l)}
}};

// sin(j pi/32), cos(j pi/32)
__device__ const double kSinTab[64] = {{
{fmt(sin_tab)}
}};
__device__ const double kCosTab[64] = {{
{fmt(cos_tab)}
}};

// ---- fixed-point tables and constants (int_math.cuh) ----
constexpr unsigned long long kTwoOverPiQ64 = {q(2 / mp.pi, 64)}ull;     // 2/pi
constexpr unsigned long long kPiOver32Q64 = {q(mp.pi / 32, 64)}ull;     // pi/32
constexpr unsigned long long k32OverPiQ59 = {q(32 / mp.pi, 59)}ull;     // 32/pi
constexpr unsigned long long kPiOver32Q128Hi = {q(mp.pi / 32, 128) >> 64}ull;   // pi/32, bits 2^-1..2^-64
constexpr unsigned long long kPiOver32Q128Lo = {q(mp.pi / 32, 128) & ((1 << 64) - 1)}ull;   // bits 2^-65..2^-128
constexpr unsigned long long kSinC3Q64 = {q(1 / fact[3], 64)}ull;
constexpr unsigned long long kSinC5Q64 = {q(1 / fact[5], 64)}ull;
constexpr unsigned long long kSinC7Q64 = {q(1 / fact[7], 64)}ull;
constexpr unsigned long long kSinC9Q64 = {q(1 / fact[9], 64)}ull;
constexpr unsigned long long kCosC2Q64 = {q(1 / fact[2], 64)}ull;
constexpr unsigned long long kCosC4Q64 = {q(1 / fact[4], 64)}ull;
constexpr unsigned long long kCosC6Q64 = {q(1 / fact[6], 64)}ull;
constexpr unsigned long long kCosC8Q64 = {q(1 / fact[8], 64)}ull;
constexpr unsigned long long kInvLn2x64Q56 = {q(64 / ln2, 56)}ull;     // 64/ln2
constexpr unsigned long long kLn2d64Q128Hi = {ln2_64_q128 >> 64}ull;   // ln2/64, bits 2^-1..2^-64
constexpr unsigned long long kLn2d64Q128Lo = {ln2_64_q128 & ((1 << 64) - 1)}ull;   // bits 2^-65..2^-128
constexpr long long kExpC2Q63 = {q(1 / fact[2], 63)}ll;
constexpr long long kExpC3Q63 = {q(1 / fact[3], 63)}ll;
constexpr long long kExpC4Q63 = {q(1 / fact[4], 63)}ll;
constexpr long long kExpC5Q63 = {q(1 / fact[5], 63)}ll;
constexpr long long kExpC6Q63 = {q(1 / fact[6], 63)}ll;

// round(sin(j pi/32) 2^62), round(cos(j pi/32) 2^62), j = 0..64
__device__ const long long kSinQ62[65] = {{
{fmt_int(sin_q62)}
}};
__device__ const long long kCosQ62[65] = {{
{fmt_int(cos_q62)}
}};
// round(2^(j/64) 2^62)
__device__ const long long kExp2Q62[64] = {{
{fmt_int(exp2_q62)}
}};

// erfcx piece k (centre k/2): coefficients of u^0 .. u^{ERFCX_DEG}, as doubles
// and in Q62
__device__ const double kErfcxTab[{ERFCX_PIECES * (ERFCX_DEG + 1)}] = {{
{fmt(erfcx_tab, 2)}
}};
__device__ const long long kErfcxQ62[{ERFCX_PIECES * (ERFCX_DEG + 1)}] = {{
{fmt_int(erfcx_q62, 2)}
}};

// Faddeeva function (faddeeva.cuh): L and Weideman's N = {WEID_N} coefficients
// a_1..a_N in Q59
constexpr int kWeidN = {WEID_N};
constexpr double kWeidL = {d(weid_L)!r};
constexpr double kInvSqrtPi = {d(1 / mp.sqrt(mp.pi))!r};
static __constant__ long long kWeidAQ59[{WEID_N}] = {{
{fmt_int(weid_q59)}
}};

}}  // namespace fp64tab
}}  // namespace ipa
"""
    with open(os.path.join(HERE, "fp64_tables.cuh"), "w") as f:
        f.write(text)


if __name__ == "__main__":
    main()
