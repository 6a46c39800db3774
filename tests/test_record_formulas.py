"""CPU checks of the readings the parameter-record kernels use (consts.cuh,
tagged.cuh, phis_consts.cuh), against the oracle and mpmath:

* the range edges through the Gaussian factor: with x = tau / sigma and gq =
  exp(-x^2/2), g(tau) = E erfc(z) / 2 is gq erfcx(z) / 2 for z >= 0 and E -
  gq erfcx(-z) / 2 for z < 0, Phi(x) = erfc(w) / 2 (w = -x / sqrt2) likewise,
  and the erfcx term is dropped below -6.25, where it does not change the sum
  in double precision; F and its derivatives then follow Sec. 3's formulas
  with 1/Gamma and 1/sigma as factors;
* the 70 entries of h_k and dh_k/dtheta_j as signed products of at most four
  factors: the table kRowSpec is read from consts.cuh and evaluated with the
  factor list its comment documents.

scipy's erfcx stands in for the kernels' table erfcx (its accuracy is tested
in test_fixed_point_special and test_gpu_math); the GPU tests compare the
device records' results with the oracle.
"""
import math
import os
import re

import numpy as np
import pytest
from scipy.special import erfcx

from oracle import ipa_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
CONSTS = os.path.join(HERE, "..", "paper_1706_01420_gb300", "csrc", "consts.cuh")
SQRT2 = math.sqrt(2.0)


def _edge(tau, Gamma, sigma):
    """(F, dF/dGamma, dF/dsigma, dF/dmu) at one edge by the record's reading."""
    rs = 1.0 / sigma
    x = tau * rs
    z = (Gamma * sigma - x) / SQRT2
    w = -x / SQRT2
    X1 = 0.0 if z < -6.25 else erfcx(abs(z))
    X2 = 0.0 if w < -6.25 else erfcx(abs(w))
    gq = math.exp(-0.5 * x * x)
    E = math.exp(-Gamma * tau + 0.5 * Gamma * Gamma * sigma * sigma)
    a = 0.5 * gq * X1
    g = E - a if z < 0 else a
    b = 0.5 * gq * X2
    Phi = 1.0 - b if w < 0 else b
    G = rs / math.sqrt(2.0 * math.pi) * gq
    rG = 1.0 / Gamma
    dg_dG = (Gamma * sigma * sigma - tau) * g - sigma * sigma * G
    dg_ds = Gamma * Gamma * sigma * g - (Gamma * sigma + x) * G
    F = (Phi - g) * rG
    return np.array([F, -(F + dg_dG) * rG, (-(x * G) - dg_ds) * rG, -g])


def _edge_mp(mp, tau, Gamma, sigma):
    """The same quantities from the closed form in 50-digit arithmetic."""
    mp.mp.dps = 50
    tau, Gamma, sigma = mp.mpf(tau), mp.mpf(Gamma), mp.mpf(sigma)
    z = (Gamma * sigma * sigma - tau) / (mp.sqrt(2) * sigma)
    g = mp.mpf(0.5) * mp.exp(-Gamma * tau + Gamma * Gamma * sigma * sigma / 2) * mp.erfc(z)
    G = mp.exp(-(tau / sigma) ** 2 / 2) / (mp.sqrt(2 * mp.pi) * sigma)
    Phi = mp.erfc(-tau / (mp.sqrt(2) * sigma)) / 2
    F = (Phi - g) / Gamma
    dg_dG = (Gamma * sigma * sigma - tau) * g - sigma * sigma * G
    dg_ds = Gamma * Gamma * sigma * g - (Gamma * sigma + tau / sigma) * G
    return [F, -(F + dg_dG) / Gamma, (-(tau / sigma) * G - dg_ds) / Gamma, -g]


# (Gamma, sigma, mu, t_lo, t_hi): the bench's range, mu off zero, a range
# starting 67 sigma before mu, wide resolution, a short range, a range wholly
# before the peak
CASES = [(0.66, 0.045, 0.0, 0.0, 15.0), (0.66, 0.045, 0.01, 0.3, 15.0), (0.66, 0.045, 0.0, -3.0, 15.0),
         (1.5, 0.3, 0.2, -1.0, 2.0), (0.2, 0.05, -0.1, 0.0, 0.5), (0.66, 0.045, 0.0, -0.3, -0.1),
         (2.0, 0.5, 0.0, -2.0, 10.0)]


@pytest.mark.parametrize("case", CASES)
def test_edges_through_the_gaussian_factor(case):
    mp = pytest.importorskip("mpmath")
    Gamma, sigma, mu, lo, hi = case
    got = _edge(hi - mu, Gamma, sigma) - _edge(lo - mu, Gamma, sigma)
    ref = np.array([float(a - b)
                    for a, b in zip(_edge_mp(mp, hi - mu, Gamma, sigma), _edge_mp(mp, lo - mu, Gamma, sigma))])
    lib = O.time_norm_grad(Gamma, sigma, mu, lo, hi)
    # every component as close to the 50-digit value as the library evaluation
    # of the same formulas, or within 1e-13: F = (Phi - g) / Gamma itself
    # cancels where the range lies before the peak (Phi and g agree there to
    # two digits), whichever way erfc is evaluated
    scale = np.abs(ref) + 1e-12 * abs(ref[0])
    err_new = np.abs(got - ref) / scale
    err_lib = np.abs(lib - ref) / scale
    assert np.all(err_new <= np.maximum(4.0 * err_lib, 1e-13)), (err_new, err_lib)


def test_dropped_erfcx_term_is_below_half_an_ulp():
    mp = pytest.importorskip("mpmath")
    # at the cut the dropped term erfc(6.25) / 2 is below half an ulp of 1 (Phi)
    # and of E (g, relative), so the sum is unchanged in double precision
    dropped = float(mp.erfc(6.25)) / 2
    assert dropped < 2.0 ** -54
    assert 1.0 - dropped == 1.0


def _row_spec():
    src = open(CONSTS).read()
    body = src[src.index("kRowSpec[kRowEntries] = {"):]
    body = re.sub(r"//[^\n]*", "", body[body.index("{") + 1:body.index("};")])
    toks = re.findall(r"kZero|kNeg \| fac\([0-9, ]+\)|fac\([0-9, ]+\)", body)
    spec = []
    for t in toks:
        if t == "kZero":
            spec.append(None)
            continue
        idx = [int(v) for v in t[t.index("(") + 1:-1].split(",")]
        spec.append((t.startswith("kNeg"), idx))
    return spec


def _factors(th):
    """The factor list of consts.cuh's comment, from the amplitude parameters."""
    x0, xe, dpa, dpe, F, dS = (float(th[i]) for i in range(4, 10))
    xa, s = 1.0 - x0 - xe, 1.0 - F
    r0, ra, re_, rF, rs = (math.sqrt(v) for v in (x0, xa, xe, F, s))
    f = [0.0] * 31
    f[0], f[1], f[2], f[3], f[4], f[5] = 1.0, s, x0, xa, xe, F
    f[6], f[7], f[8], f[9] = ra, re_, r0, rF * rs
    f[10], f[11], f[12] = 0.5 / (ra * re_), 0.5 / (r0 * ra), 0.5 / (r0 * re_)
    f[13], f[14], f[15] = 0.5 / ra, 0.5 / re_, 0.5 / r0
    f[16] = (1.0 - 2.0 * F) * 0.5 / (rF * rs)
    f[17], f[18] = xa - xe, xa - x0
    for i, a in enumerate((dpe - dpa, dpa, dpe, dpa - dS, dpe - dS, dS)):
        f[19 + i], f[25 + i] = math.sin(a), math.cos(a)
    return f


@pytest.mark.parametrize("th", [[0, 0, 0, 0, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3],
                                [0, 0, 0, 0, 0.3, 0.4, -1.0, 0.5, 0.2, 2.0],
                                [0, 0, 0, 0, 0.1, 0.1, 0.3, -2.5, 0.6, -0.7]])
def test_angular_factor_table(th):
    spec = _row_spec()
    assert len(spec) == 70
    f = _factors(th)
    vals = []
    for e in spec:
        if e is None:
            vals.append(0.0)
            continue
        neg, idx = e
        assert len(idx) <= 4 and all(0 <= i < 31 for i in idx)
        v = 1.0
        for i in idx:
            v *= f[i]
        vals.append(-v if neg else v)
    h, dh = np.array(vals[:10]), np.array(vals[10:]).reshape(10, 6)
    np.testing.assert_allclose(h, O.amplitude_coeffs(th), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(dh, O.amplitude_coeffs_grad(th), rtol=1e-13, atol=1e-15)
