"""CPU emulation of the device Faddeeva function (faddeeva.cuh) with the
generated coefficients (fp64_tables.cuh), against mpmath's complex erfc.

The emulation repeats the kernel's operation order in FP64 (without FMA
contraction), so it checks the coefficient table, the choice of L and N and
the algebra of the evaluation before any GPU run; the GPU test compares the
device results themselves with scipy.
"""
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(HERE, "..", "paper_1706_01420_gb300", "csrc", "fp64_tables.cuh")


@pytest.fixture(scope="module")
def weid():
    src = open(TABLES).read()
    L = float(re.search(r"kWeidL = ([0-9.eE+-]+);", src).group(1))
    n = int(re.search(r"kWeidN = (\d+);", src).group(1))
    blk = re.search(r"kWeidA\[\d+\] = \{(.*?)\};", src, re.S).group(1)
    a = [float(v) for v in blk.replace("\n", " ").split(",") if v.strip()]
    isp = float(re.search(r"kInvSqrtPi = ([0-9.eE+-]+);", src).group(1))
    assert len(a) == n == 40
    return L, a, isp


def _w(weid, x, y):
    L, a, isp = weid
    dr = L + y
    inv = 1.0 / (dr * dr + x * x)
    er, ei = dr * inv, x * inv
    nr = L - y
    Zr, Zi = nr * er - x * ei, nr * ei + x * er
    pr, pi = a[-1], 0.0
    for k in range(len(a) - 2, -1, -1):
        t = pr * Zr + (-pi * Zi + a[k])
        pi = pr * Zi + pi * Zr
        pr = t
    tr = 2.0 * (pr * er - pi * ei) + isp
    ti = 2.0 * (pr * ei + pi * er)
    return complex(tr * er - ti * ei, tr * ei + ti * er)


def test_emulated_faddeeva_matches_mpmath(weid):
    mp = pytest.importorskip("mpmath")
    worst = 0.0
    with mp.workdps(30):      # local precision: other tests set the global one
        for x in np.linspace(-8, 8, 33):
            for y in (0.0, 1e-3, 0.3, 1.0, 2.5, 6.3, 12.0, 50.0, 1e3, 1e6):
                z = mp.mpc(x, y)
                ref = complex(mp.exp(-z * z) * mp.erfc(-1j * z))
                worst = max(worst, abs(_w(weid, x, y) - ref) / abs(ref))
    assert worst < 1.5e-15, worst


def test_constants(weid):
    """L = 2^(-1/4) sqrt(40); a_n decay (the series is truncated where they reach 1e-15)."""
    L, a, isp = weid
    assert L == pytest.approx(2 ** -0.25 * 40 ** 0.5, rel=1e-15)
    assert isp == pytest.approx(np.pi ** -0.5, rel=1e-16)
    assert max(abs(v) for v in a[-4:]) < 2e-14
