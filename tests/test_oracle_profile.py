"""Pins of the oracle's error analysis (oracle/profile.py): HESSE covariance
and MINOS profile-likelihood intervals.

* HESSE equals the closed-form second derivative of the NLL of a truncated
  exponential (the 1D model as sigma -> 0 without background), and the second
  differences of the NLL itself (no gradient) for two free parameters;
* MINOS with one free parameter equals a direct bisection of
  NLL(x) = NLL_min + 1/2; with a second free parameter it equals a profile
  computed by golden-section minimisation over that parameter; for a large
  sample it approaches the HESSE error; an interval that runs into a limit is
  reported at the limit.
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth


@pytest.fixture(scope="module")
def P():
    from oracle import profile
    return profile


def _bisect(f, a, b, n=200):
    fa = f(a)
    for _ in range(n):
        m = 0.5 * (a + b)
        fm = f(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def _golden_min(f, a, b, n=90):
    g = (math.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(n):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return min(fc, fd)


def test_hesse_exponential_closed_form(oracle, P):
    """sigma = 1e-4, mu = 0, f_b = 0: P(t) -> Gamma e^{-Gamma t} / D(Gamma),
    D = e^{-Gamma a} - e^{-Gamma b}; d2 NLL / dGamma2 = N / Gamma^2 + N (D'' D - D'^2) / D^2."""
    a, b = 0.3, 15.0
    truth = {"Gamma": 0.66, "sigma": 1e-4, "mu": 0.0, "f_b": 0.0}
    t = synth.events_1d(20000, 5, t_lo=a, t_hi=b, truth=truth)
    m = oracle.Model("1d", a, b)
    G = 0.7
    C, err, corr, H = P.hesse(m, {"t": t}, [G, 1e-4, 0.0, 0.0], [0])
    N = t.size
    D = math.exp(-G * a) - math.exp(-G * b)
    D1 = -a * math.exp(-G * a) + b * math.exp(-G * b)
    D2 = a * a * math.exp(-G * a) - b * b * math.exp(-G * b)
    h_exact = N / G ** 2 + N * (D2 * D - D1 * D1) / (D * D)
    assert H[0, 0] == pytest.approx(h_exact, rel=1e-6)
    assert C[0, 0] == pytest.approx(1.0 / h_exact, rel=1e-6)
    assert err[0] == pytest.approx(h_exact ** -0.5, rel=1e-6)


def test_hesse_matches_second_differences_of_the_nll(oracle, P):
    m = oracle.Model("1d", 0.3, 15.0)
    ev = {"t": synth.events_1d(10000, 6)}
    th = np.array([0.67, 0.045, 0.0, 0.09])
    free = [0, 3]
    C, err, corr, H = P.hesse(m, ev, th, free)
    hs = [1e-3 * math.sqrt(C[j, j]) for j in free]
    Hn = np.zeros((2, 2))
    for x, (i, hi) in enumerate(zip(free, hs)):
        for y, (j, hj) in enumerate(zip(free, hs)):
            def f(si, sj):
                tt = th.copy()
                tt[i] += si * hi
                tt[j] += sj * hj
                return oracle.nll(m, ev, tt)
            Hn[x, y] = (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * hi * hj)
    np.testing.assert_allclose(H, Hn, rtol=2e-4)
    assert np.allclose(corr, corr.T) and np.allclose(np.diag(corr), 1.0)
    assert abs(corr[0, 1]) < 1.0


def test_minos_single_parameter_is_the_nll_crossing(oracle, P):
    m = oracle.Model("1d", 0.3, 15.0)
    ev = {"t": synth.events_1d(3000, 7)}
    th0 = np.array([0.66, 0.045, 0.0, 0.1])
    r = oracle.fit(m, ev, th0, [0], tol=1e-12)
    (elo, ehi), st = P.minos(m, ev, r.theta, r.nll, [0], 0, r.err[0])
    assert st == ("OK", "OK")

    def excess(x):
        tt = r.theta.copy()
        tt[0] = x
        return oracle.nll(m, ev, tt) - r.nll - 0.5

    s = r.err[0]
    xl = _bisect(excess, r.theta[0] - 5 * s, r.theta[0])
    xh = _bisect(excess, r.theta[0], r.theta[0] + 5 * s)
    assert abs(elo - (xl - r.theta[0])) < 1e-9 * s
    assert abs(ehi - (xh - r.theta[0])) < 1e-9 * s
    assert elo < 0 < ehi


def test_minos_profiles_out_the_other_parameter(oracle, P):
    m = oracle.Model("1d", 0.3, 15.0)
    ev = {"t": synth.events_1d(2000, 8)}
    th0 = np.array([0.66, 0.045, 0.0, 0.1])
    free = [0, 3]
    r = oracle.fit(m, ev, th0, free, lo=[0.1, 0, -1, 0.0], hi=[3.0, 1, 1, 1.0], tol=1e-12)
    (elo, ehi), st = P.minos(m, ev, r.theta, r.nll, free, 0, r.err[0], lo=[0.1, 0, -1, 0.0], hi=[3.0, 1, 1, 1.0])

    def excess(x):
        def nll_fb(fb):
            tt = r.theta.copy()
            tt[0], tt[3] = x, fb
            return oracle.nll(m, ev, tt)
        return _golden_min(nll_fb, max(0.0, r.theta[3] - 0.2), r.theta[3] + 0.2) - r.nll - 0.5

    s = r.err[0]
    xh = _bisect(excess, r.theta[0], r.theta[0] + 4 * s, n=60)
    xl = _bisect(excess, r.theta[0] - 4 * s, r.theta[0], n=60)
    assert abs(ehi - (xh - r.theta[0])) < 1e-6 * s
    assert abs(elo - (xl - r.theta[0])) < 1e-6 * s
    # the profile is wider than the slice at fixed f_b
    (slo, shi), _ = P.minos(m, ev, r.theta, r.nll, [0], 0, r.err[0])
    assert ehi > shi and elo < slo


def test_minos_approaches_hesse_for_a_large_sample(oracle, P):
    m = oracle.Model("1d", 0.3, 15.0)
    ev = {"t": synth.events_1d(20000, 9)}
    free = [0, 3]
    r = oracle.fit(m, ev, np.array([0.66, 0.045, 0.0, 0.1]), free, tol=1e-12)
    C, err, corr, H = P.hesse(m, ev, r.theta, free)
    (elo, ehi), st = P.minos(m, ev, r.theta, r.nll, free, 0, err[0], tol=1e-8)
    assert st == ("OK", "OK")
    # the asymmetry is of order 1/sqrt(N) of the error
    assert abs(-elo / err[0] - 1) < 0.04 and abs(ehi / err[0] - 1) < 0.04, (elo, ehi, err[0])
    assert abs(-elo / err[0] - 1) > 1e-4      # the interval is not HESSE's copy


def test_minos_interval_at_a_limit(oracle, P):
    """No background in the sample: f_b's lower interval runs into f_b = 0."""
    m = oracle.Model("1d", 0.3, 15.0)
    truth = {"Gamma": 0.66, "sigma": 0.045, "mu": 0.0, "f_b": 0.0}
    ev = {"t": synth.events_1d(2000, 10, truth=truth)}
    lo, hi = [0.1, 0.0, -1.0, 0.0], [3.0, 1.0, 1.0, 1.0]
    free = [0, 3]
    r = oracle.fit(m, ev, np.array([0.66, 0.045, 0.0, 0.02]), free, lo=lo, hi=hi, tol=1e-10)
    C, err, corr, H = P.hesse(m, ev, r.theta, free)
    (elo, ehi), st = P.minos(m, ev, r.theta, r.nll, free, 3, max(err[3], 1e-3), lo=lo, hi=hi)
    assert r.theta[3] < 0.5 * err[3]          # the minimum sits within half an error of the limit
    assert st[0] == "LIMIT" and elo == pytest.approx(-r.theta[3], abs=1e-15)
    assert st[1] == "OK" and ehi > 0
