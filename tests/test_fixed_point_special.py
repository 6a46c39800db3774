"""Bit-exact CPU emulation of the fixed-point special functions of the
likelihood kernels, against mpmath:

* erfcx_poly_q (int_math.cuh): the piecewise erfcx on [0, 6.25] with x in Q60,
  u in Q63 and the Q62 coefficients of fp64_tables.cuh, Horner's rule with
  floored 64 x 64 -> 128-bit high halves, one rounding to double;
* the Faddeeva function's Horner sum in Z (faddeeva.cuh, Weideman's rational
  approximation): Z in Q62, partial sums in Q59 with the kernel's bias
  correction, the FP64 parts repeated in the kernel's operation order (without
  FMA contraction).

The integer arithmetic is emulated exactly (Python integers: a floored high
half is (a b) >> 64), so these tests check the tables, the fixed-point
formats (no overflow, the claimed error) and the algebra before any GPU run;
test_gpu_math and test_gpu_tagged compare the device results with scipy.
"""
import os
import re
import struct

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(HERE, "..", "paper_1706_01420_gb300", "csrc", "fp64_tables.cuh")
I64 = 1 << 63


def _ints(src, name):
    blk = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
    return [int(v.strip().rstrip("l")) for v in blk.replace("\n", " ").split(",") if v.strip()]


@pytest.fixture(scope="module")
def tables():
    src = open(TABLES).read()
    ex = _ints(src, "kErfcxQ62")
    wa = _ints(src, "kWeidAQ59")
    L = float(re.search(r"kWeidL = ([0-9.eE+-]+);", src).group(1))
    isp = float(re.search(r"kInvSqrtPi = ([0-9.eE+-]+);", src).group(1))
    pieces = int(re.search(r"kErfcxPieces = (\d+);", src).group(1))
    coeffs = int(re.search(r"kErfcxCoeffs = (\d+);", src).group(1))
    assert len(ex) == pieces * coeffs and len(wa) == 40
    return ex, pieces, coeffs, wa, L, isp


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _wrap(v):
    """Two's complement wrap to a signed 64-bit value (the kernel's casts)."""
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= I64 else v


def _mulhi(a, b):
    assert -I64 <= a < I64 and -I64 <= b < I64
    return (a * b) >> 64


def _shift_nb(M, sh):
    if sh >= 0:
        return (M << (sh & 63)) & ((1 << 64) - 1)
    return M >> ((-sh) & 63) if sh > -64 else 0


def _to_q62(x):
    """to_q62_nb: x 2^62 truncated toward zero, for |x| < 2."""
    b = _bits(x) & ((1 << 64) - 1)
    M = (b & ((1 << 52) - 1)) | (1 << 52)
    v = _shift_nb(M, ((b >> 52) & 0x7FF) - 1023 + 10)
    assert v < I64
    return -v if b >> 63 else v


def _q_to_double(v, frac_bits):
    return v / (1 << frac_bits)          # correctly rounded, as q62_to_double_nb


def erfcx_emulated(tables, x):
    """erfcx_poly_q."""
    ex, pieces, coeffs = tables[:3]
    b = _bits(x) & 0x7FFFFFFFFFFFFFFF
    b = min(b, 0x4019000000000000)                          # 6.25
    M = (b & ((1 << 52) - 1)) | (1 << 52)
    X = _shift_nb(M, (b >> 52) - 1023 + 8)
    assert X < I64
    k = min((X + (1 << 58)) >> 59, pieces - 1)
    u = _wrap((X - (k << 59)) << 3)
    assert abs(u) <= 1 << 61
    c = ex[k * coeffs:(k + 1) * coeffs]
    v = c[-1]
    for i in range(coeffs - 2, -1, -1):
        v = c[i] + _wrap(_mulhi(v, u) << 1)
        assert abs(v) < 3 << 61                            # |v| < 1.5 in Q62
    return _q_to_double(v, 62)


def faddeeva_emulated(tables, xs, y):
    """faddeeva_uhp: evaluated at |x|, conjugated for x < 0."""
    wa, L, isp = tables[3:]
    x = abs(xs)
    dr = L + y
    inv = 1.0 / (dr * dr + x * x)
    er, ei = dr * inv, x * inv
    nr = L - y
    Zr, Zi = nr * er - x * ei, nr * ei + x * er
    zr, zi = _to_q62(Zr), _to_q62(Zi)
    qr, qi = wa[-1], 0
    for k in range(len(wa) - 2, -1, -1):
        t = wa[k] + _wrap((_mulhi(qr, zr) - _mulhi(qi, zi)) << 2)
        qi = _wrap((_mulhi(qr, zi) + _mulhi(qi, zr) + 1) << 2)
        qr = t
        assert abs(qr) < 16 << 59 and abs(qi) < 16 << 59
    pr, pi = _q_to_double(qr, 59), _q_to_double(qi, 59)
    tr = 2.0 * (pr * er - pi * ei) + isp
    ti = 2.0 * (pr * ei + pi * er)
    wi = tr * ei + ti * er
    return complex(tr * er - ti * ei, -wi if np.signbit(xs) else wi)


def test_erfcx_fixed_point_matches_mpmath(tables):
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.uniform(0.0, 6.25, 3000), np.arange(0, 13) / 2, np.arange(0, 13) / 2 + 0.25,
                         [1e-300, 5e-324, 2.0 ** -60, 6.25, np.nextafter(6.25, 0)]])
    worst = 0.0
    with mp.workdps(30):
        for x in xs:
            ref = float(mp.exp(mp.mpf(x) ** 2) * mp.erfc(mp.mpf(x)))
            worst = max(worst, abs(erfcx_emulated(tables, float(x)) - ref) / ref)
    # the interpolants' own error (~1e-16) plus the final rounding; the fixed
    # point adds below 2e-17
    assert worst < 4e-16, worst


def test_erfcx_fixed_point_outside_the_range_is_finite(tables):
    """Inputs the callers select away (above 6.25, infinite, NaN, negative)
    still run in range: no overflow, a finite value."""
    for x in (6.2500001, 7.0, 1e300, float("inf"), float("nan"), -0.0, -3.0):
        assert np.isfinite(erfcx_emulated(tables, x))


def test_faddeeva_fixed_point_matches_mpmath(tables):
    mp = pytest.importorskip("mpmath")
    worst = 0.0
    with mp.workdps(30):
        for x in np.linspace(-8, 8, 33):
            for y in (0.0, 1e-3, 0.3, 1.0, 2.5, 6.3, 12.0, 50.0, 1e3, 1e6):
                z = mp.mpc(x, y)
                ref = complex(mp.exp(-z * z) * mp.erfc(-1j * z))
                worst = max(worst, abs(faddeeva_emulated(tables, x, y) - ref) / abs(ref))
    assert worst < 1.5e-15, worst


def test_faddeeva_fixed_point_at_the_tagged_model_arguments(tables):
    """The arguments of the tagged kernel's slow branch: x = +-beta (beta =
    Dm sigma / sqrt 2 for Dm in [10, 25], sigma in [0.02, 0.06]), 0 <= y <= 7."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(12)
    worst = 0.0
    with mp.workdps(30):
        for _ in range(400):
            beta = rng.uniform(10, 25) * rng.uniform(0.02, 0.06) / np.sqrt(2.0)
            x = beta if rng.uniform() < 0.5 else -beta
            y = rng.uniform(0.0, 7.0)
            z = mp.mpc(x, y)
            ref = complex(mp.exp(-z * z) * mp.erfc(-1j * z))
            worst = max(worst, abs(faddeeva_emulated(tables, x, y) - ref) / abs(ref))
    assert worst < 1e-15, worst


def test_fixed_point_tables_round_the_generator_values(tables):
    """The Q62 / Q59 tables are the rounded exact values: a_1 of Weideman's
    series and the constant term of erfcx's first piece, erfcx(0) = 1."""
    ex, pieces, coeffs, wa = tables[:4]
    assert abs(ex[0] - (1 << 62)) <= 1 << 12          # erfcx(0) = 1 to the interpolant's accuracy
    assert abs(ex[1] / 2 ** 62 + 2 / np.sqrt(np.pi)) < 1e-13   # erfcx'(0) = -2/sqrt(pi)
    assert sum(abs(a) for a in wa) < 13 << 59


def test_weideman_constants(tables):
    """L = 2^(-1/4) sqrt(40); 1/sqrt(pi); the a_n decay (the series is truncated
    where they reach 1e-15)."""
    wa, L, isp = tables[3:]
    assert L == pytest.approx(2 ** -0.25 * 40 ** 0.5, rel=1e-15)
    assert isp == pytest.approx(np.pi ** -0.5, rel=1e-16)
    assert max(abs(v) for v in wa[-4:]) < 2e-14 * 2 ** 59
