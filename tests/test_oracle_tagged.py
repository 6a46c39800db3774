"""Pins of the oracle's flavour-tagged decay-time model (oracle/tagged.py).

* the complex convolution g(tau; Gamma - i Dm) equals brute-force quadrature
  of e^{-Gamma u} (cos, sin)(Dm u) G(tau - u) (both parts), reduces to the
  real decay-time convolution for Dm = 0, and to e^{-z tau} as sigma -> 0;
* the PDF integrates to 1 over t and both tags; S >= 0 and S <= the
  generator's envelope on a dense grid;
* phi_s = 0 makes the model tag-blind and equal to half the 1D model with
  Gamma_L; the gradient equals central finite differences of the NLL;
* generated toys: exact counts, the tag asymmetry follows the model's
  oscillation, a Newton fit (mistag held) recovers the generating parameters.
"""
import math

import numpy as np
import pytest
from scipy import integrate

TRUTH = np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.8, 0.3])


@pytest.fixture(scope="module")
def T():
    from oracle import tagged
    return tagged


@pytest.mark.parametrize("Dm", [17.77, 0.5])
@pytest.mark.parametrize("tau", [-0.08, -0.01, 0.0, 0.03, 0.3, 2.5])
def test_complex_convolution_matches_quadrature(oracle, T, tau, Dm):
    G, s = 0.66, 0.045
    lo, hi = max(0.0, tau - 14 * s), tau + 14 * s
    re = integrate.quad(lambda u: math.exp(-G * u) * math.cos(Dm * u) * oracle.gauss(tau - u, s), lo, hi,
                        limit=500, epsabs=0, epsrel=1e-13)[0]
    im = integrate.quad(lambda u: math.exp(-G * u) * math.sin(Dm * u) * oracle.gauss(tau - u, s), lo, hi,
                        limit=500, epsabs=0, epsrel=1e-13)[0]
    g = T.conv_c(tau, complex(G, -Dm), s)[0]
    assert abs(g.real - re) <= 2e-15 and abs(g.imag - im) <= 2e-15


def test_complex_convolution_limits(oracle, T):
    tau = np.linspace(-0.2, 10, 301)
    g = T.conv_c(tau, complex(0.66, 0.0), 0.045)
    np.testing.assert_allclose(g.real, oracle.time_conv(tau, 0.66, 0.045), rtol=1e-14, atol=1e-300)
    assert np.all(g.imag == 0.0)
    z = complex(0.66, -17.77)
    tp = np.linspace(0.5, 5, 50)
    small = T.conv_c(tp, z, 1e-5)
    np.testing.assert_allclose(small, np.exp(-z * tp), rtol=1e-7)


@pytest.mark.parametrize("theta", [TRUTH, np.array([1.2, 0.08, 0.02, 0.3, -0.1, 5.0, -2.0, 0.1]),
                                   np.array([0.5, 0.03, -0.01, 0.0, 0.2, 25.0, 1.57, 0.45])])
def test_pdf_integrates_to_one(oracle, T, theta):
    m = oracle.Model("tag", 0.0, 15.0)
    tot = 0.0
    for q in (-1.0, 1.0):
        f = lambda t: T.pdf(m, {"t": np.array([t]), "q": np.array([q])}, theta)[0]
        tot += integrate.quad(f, 0.0, 15.0, limit=4000, points=[0.05, 0.2, 1.0, 3.0], epsrel=1e-12)[0]
    assert abs(tot - 1.0) < 1e-10


def test_positive_and_below_envelope(oracle, T):
    rng = np.random.default_rng(1)
    m = oracle.Model("tag", -0.3, 12.0)
    t = np.linspace(-0.3, 12.0, 4001)
    for _ in range(40):
        th = np.array([rng.uniform(0.3, 2.0), rng.uniform(0.02, 0.2), rng.uniform(-0.05, 0.05), 0.1,
                       rng.uniform(-0.3, 0.3), rng.uniform(0.3, 30.0), rng.uniform(-3.1, 3.1),
                       rng.uniform(0.0, 0.5)])
        env = T.envelope(m, th)
        for q in (-1.0, 1.0):
            S, _ = T.signal(m, {"t": t, "q": np.full_like(t, q)}, th)
            assert S.min() > -1e-15 and S.max() <= env * (1 + 1e-12)


def test_phi_zero_is_tag_blind_1d_model(oracle, T):
    th = TRUTH.copy()
    th[6] = 0.0
    m = oracle.Model("tag", 0.0, 15.0)
    t = np.linspace(0.0, 15.0, 200)
    pp = T.pdf(m, {"t": t, "q": np.ones_like(t)}, th)
    pm = T.pdf(m, {"t": t, "q": -np.ones_like(t)}, th)
    np.testing.assert_array_equal(pp, pm)
    p1 = oracle.pdf(oracle.Model("1d", 0.0, 15.0), {"t": t}, [th[0] + th[4] / 2, th[1], th[2], th[3]])
    np.testing.assert_allclose(pp, 0.5 * p1, rtol=1e-14)


def test_gradient_matches_finite_differences(oracle, T):
    m = oracle.Model("tag", 0.0, 15.0)
    rng = np.random.default_rng(2)
    n = 3000
    ev = {"t": rng.uniform(0.0, 15.0, n) ** 1.0, "q": np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0),
          "w": rng.normal(1.0, 0.2, n)}
    th = TRUTH + np.array([0.01, 0.002, 0.001, 0.02, 0.01, 0.05, 0.05, 0.01])
    f, g = oracle.nll_grad(m, ev, th)
    for j in range(8):
        h = 1e-5 * max(abs(th[j]), 1e-2)
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (oracle.nll(m, ev, tp) - oracle.nll(m, ev, tm)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(abs(g[j]), 1.0), (j, fd, g[j])


def test_toys_counts_and_oscillation(oracle, T):
    m = oracle.Model("tag", 0.0, 15.0)
    ev = oracle.toy_one(m, TRUTH, 3, 0, 60000, 500)
    assert ev["t"].size == 60500 and set(np.unique(ev["q"])) == {-1.0, 1.0}
    # signal tag asymmetry in time bins follows the model: compare counts with
    # the model's integral per bin and tag (chi^2)
    edges = np.linspace(0.0, 2.0, 41)
    chi2, nb = 0.0, 0
    for q in (-1.0, 1.0):
        sel = ev["q"][:60000] == q
        obs = np.histogram(ev["t"][:60000][sel], edges)[0]
        th = TRUTH.copy()
        th[3] = 0.0
        p = np.array([integrate.quad(lambda x: T.pdf(m, {"t": np.array([x]), "q": np.array([q])}, th)[0],
                                     a, b, epsrel=1e-10)[0] for a, b in zip(edges[:-1], edges[1:])])
        exp = 60000 * p
        chi2 += float(np.sum((obs - exp) ** 2 / exp))
        nb += len(exp)
    assert chi2 < nb + 5 * math.sqrt(2 * nb)


def test_fit_recovers_truth(oracle, T):
    """The mistag omega is held at its calibrated value (the tagged term only
    measures (1 - 2 omega) sin phi_s, so omega and phi_s are degenerate)."""
    m = oracle.Model("tag", 0.0, 15.0)
    ev = oracle.toy_one(m, TRUTH, 4, 0, 36000, 4000)
    free = [0, 3, 4, 5, 6]
    lo = np.array([0.3, 0.01, -0.1, 0.0, -0.5, 10.0, -3.1, 0.0])
    hi = np.array([1.5, 0.2, 0.1, 0.5, 0.5, 25.0, 3.1, 0.5])
    r = oracle.fit(m, ev, TRUTH * 1.01, free, lo=lo, hi=hi, tol=1e-7, max_iter=60)
    assert r.status == "CONVERGED"
    pulls = (r.theta[free] - TRUTH[free]) / r.err[free]
    assert np.all(np.abs(pulls) < 4.5), pulls
