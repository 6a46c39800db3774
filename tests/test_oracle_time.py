"""Pins of the oracle's decay-time PDF against mathematics it does not use itself.

* the closed-form convolution vs brute-force numerical convolution
  (adaptive quadrature, and a trapezoid rule on a tiny grid that converges as h^2);
* the sigma -> 0 limit vs the textbook exponential, and the normalisation in
  that limit vs the analytic exponential integral printed in Sec. 3 (Example 1);
* the analytic normalisation I_T vs adaptive quadrature of the PDF;
* the derivatives vs central finite differences.
"""
import math

import numpy as np
import pytest
from scipy import integrate

GAMMA, SIGMA = 0.66, 0.045


def brute_conv(tau, Gamma, sigma):
    """int_0^inf exp(-Gamma s) N(tau - s; 0, sigma) ds by adaptive quadrature (no erfc)."""
    f = lambda s: math.exp(-Gamma * s) * math.exp(-0.5 * ((tau - s) / sigma) ** 2) / (math.sqrt(2 * math.pi) * sigma)
    lo, hi = max(0.0, tau - 12 * sigma), max(0.0, tau + 12 * sigma)
    core = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0] if hi > lo else 0.0
    return core


@pytest.mark.parametrize("tau", [-0.15, -0.05, 0.0, 0.01, 0.03, 0.1, 0.3, 2.0, 9.0])
@pytest.mark.parametrize("Gamma,sigma", [(0.66, 0.045), (1.5, 0.1), (0.3, 0.02)])
def test_conv_matches_quadrature(oracle, tau, Gamma, sigma):
    ref = brute_conv(tau, Gamma, sigma)
    got = float(oracle.time_conv(tau, Gamma, sigma))
    assert got == pytest.approx(ref, rel=1e-11, abs=1e-300)


def test_conv_matches_trapezoid_grid(oracle):
    """Tiny-grid trapezoid convolution converges to the closed form at rate h^2."""
    tau = 0.05
    errs = []
    for h in (SIGMA / 50, SIGMA / 100, SIGMA / 200):
        s = np.arange(0.0, tau + 12 * SIGMA + h / 2, h)
        y = np.exp(-GAMMA * s) * np.exp(-0.5 * ((tau - s) / SIGMA) ** 2) / (math.sqrt(2 * math.pi) * SIGMA)
        trap = h * (y.sum() - 0.5 * (y[0] + y[-1]))
        errs.append(abs(trap - float(oracle.time_conv(tau, GAMMA, SIGMA))))
    assert errs[2] < 1e-5
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def test_sigma_to_zero_is_exponential(oracle):
    tau = np.array([0.05, 0.3, 1.0, 5.0, 14.0])
    got = oracle.time_conv(tau, GAMMA, 1e-7)
    np.testing.assert_allclose(got, np.exp(-GAMMA * tau), rtol=1e-12)


@pytest.mark.parametrize("k,mmin,mmax", [(-0.66, 0.3, 15.0), (-1.2, 0.5, 4.0), (-0.25, 1.0, 9.0)])
def test_normalisation_reduces_to_sec3_exponential_integral(oracle, k, mmin, mmax):
    """Sec. 3 prints integral_exp = (exp(k Mmax) - exp(k Mmin)) / k for exp(k m); with
    Gamma = -k and a negligible resolution, I_T must equal it."""
    paper = (math.exp(k * mmax) - math.exp(k * mmin)) / k
    got = oracle.time_norm(-k, 1e-7, 0.0, mmin, mmax)
    assert got == pytest.approx(paper, rel=1e-12)


@pytest.mark.parametrize("t_lo,t_hi", [(0.3, 15.0), (0.0, 15.0), (-0.2, 15.0), (0.0, 0.5)])
@pytest.mark.parametrize("Gamma,sigma,mu", [(0.66, 0.045, 0.0), (1.1, 0.08, 0.02), (0.4, 0.03, -0.01)])
def test_normalisation_matches_quadrature(oracle, t_lo, t_hi, Gamma, sigma, mu):
    f = lambda t: float(oracle.time_conv(t - mu, Gamma, sigma))
    pts = [p for p in (mu, mu + 0.1, mu + 0.5, mu + 2.0) if t_lo < p < t_hi]
    ref = integrate.quad(f, t_lo, t_hi, points=pts or None, epsabs=0, epsrel=1e-13, limit=400)[0]
    assert oracle.time_norm(Gamma, sigma, mu, t_lo, t_hi) == pytest.approx(ref, rel=1e-12)


def test_mixture_1d_integrates_to_one(oracle):
    m = oracle.Model("1d", 0.3, 15.0)
    th = [0.66, 0.045, 0.0, 0.1]
    f = lambda t: float(oracle.pdf(m, {"t": np.array([t])}, th)[0])
    val = integrate.quad(f, 0.3, 15.0, points=[0.5, 2.0], epsabs=0, epsrel=1e-13, limit=400)[0]
    assert val == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("tau", [-0.05, 0.0, 0.02, 0.2, 3.0])
def test_conv_derivatives_vs_finite_differences(oracle, tau):
    g, dG, dS, dT = (float(v) for v in oracle.time_conv_grad(tau, GAMMA, SIGMA))
    h = 1e-6
    fd = lambda fn, x: (fn(x + h * max(1, abs(x))) - fn(x - h * max(1, abs(x)))) / (2 * h * max(1, abs(x)))
    assert dG == pytest.approx(fd(lambda G: float(oracle.time_conv(tau, G, SIGMA)), GAMMA), rel=1e-6, abs=1e-9)
    hs = 1e-7
    fds = (float(oracle.time_conv(tau, GAMMA, SIGMA + hs)) - float(oracle.time_conv(tau, GAMMA, SIGMA - hs))) / (2 * hs)
    assert dS == pytest.approx(fds, rel=1e-6, abs=1e-8)
    ht = 1e-7
    fdt = (float(oracle.time_conv(tau + ht, GAMMA, SIGMA)) - float(oracle.time_conv(tau - ht, GAMMA, SIGMA))) / (2 * ht)
    assert dT == pytest.approx(fdt, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("t_lo,t_hi,mu", [(0.0, 15.0, 0.0), (0.3, 15.0, 0.01), (-0.1, 10.0, -0.02)])
def test_normalisation_derivatives_vs_finite_differences(oracle, t_lo, t_hi, mu):
    I, dG, dS, dM = oracle.time_norm_grad(GAMMA, SIGMA, mu, t_lo, t_hi)
    assert I == pytest.approx(oracle.time_norm(GAMMA, SIGMA, mu, t_lo, t_hi), rel=1e-15)
    for j, ana in ((0, dG), (1, dS), (2, dM)):
        p = [GAMMA, SIGMA, mu]
        h = 1e-6 * max(abs(p[j]), 1e-2)
        pp, pm = list(p), list(p)
        pp[j] += h
        pm[j] -= h
        fd = (oracle.time_norm(*pp, t_lo, t_hi) - oracle.time_norm(*pm, t_lo, t_hi)) / (2 * h)
        assert ana == pytest.approx(fd, rel=1e-6, abs=1e-9)
