"""Pins of the oracle's NLL and analytic gradient.

* gradient vs central finite differences of the NLL (1e-6 relative);
* invariants of the weighted sum: unit weights equal the unweighted NLL, scaling
  the weights scales NLL and gradient, splitting the sample adds up;
* the correctly rounded sum vs an exact rational sum.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

TH1 = np.array([0.66, 0.045, 0.0, 0.1])
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])


def _fd_grad(oracle, m, ev, th, rel=1e-5):
    """Central differences and their rounding noise |NLL| * 4 eps / h."""
    g = np.zeros(th.size)
    noise = np.zeros(th.size)
    f0 = abs(oracle.nll(m, ev, th))
    for j in range(th.size):
        h = rel * max(abs(th[j]), 0.05)
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        g[j] = (oracle.nll(m, ev, tp) - oracle.nll(m, ev, tm)) / (2 * h)
        noise[j] = f0 * 4 * np.finfo(float).eps / h
    return g, noise


@pytest.mark.parametrize("kind,t_lo", [("1d", 0.3), ("1d", 0.0), ("4d", 0.0)])
def test_gradient_vs_finite_differences(oracle, kind, t_lo):
    m = oracle.Model(kind, t_lo, 15.0)
    th = (TH1 if kind == "1d" else TH4).copy()
    th[2] = 0.004                        # off-centre resolution offset: exercises dmu
    ev = synth.events_4d(3000, seed=1, t_lo=t_lo, weighted=True) if kind == "4d" else \
        {"t": synth.events_1d(3000, seed=1, t_lo=t_lo), "w": synth.weights(3000, 2)}
    _, g = oracle.nll_grad(m, ev, th)
    fd, noise = _fd_grad(oracle, m, ev, th)
    _, terms = oracle.nll_grad_terms(m, ev, th)
    scale = np.abs(terms).sum(axis=1)
    # 1e-6 relative to the gradient (or to 1e-3 of the sum of |per-event terms| where the
    # gradient cancels), plus the rounding noise of the differences: on [0.3, 15] ps the
    # resolution parameters carry almost no information and their gradient is ~1e-8.
    assert np.all(np.abs(g - fd) <= 1e-6 * np.maximum(np.abs(g), 1e-3 * scale) + noise)


def test_weights_invariants(oracle):
    m = oracle.Model("4d", 0.0, 15.0)
    ev = synth.events_4d(2000, seed=4)
    f0, g0 = oracle.nll_grad(m, ev, TH4)
    ev1 = dict(ev, w=np.ones(2000))
    f1, g1 = oracle.nll_grad(m, ev1, TH4)
    assert f1 == f0 and np.array_equal(g1, g0)
    ev2 = dict(ev, w=np.full(2000, 2.0))
    f2, g2 = oracle.nll_grad(m, ev2, TH4)
    assert f2 == 2 * f0 and np.array_equal(g2, 2 * g0)
    a = {k: v[:700] for k, v in ev.items()}
    b = {k: v[700:] for k, v in ev.items()}
    fa, ga = oracle.nll_grad(m, a, TH4)
    fb, gb = oracle.nll_grad(m, b, TH4)
    assert fa + fb == pytest.approx(f0, rel=1e-15)
    np.testing.assert_allclose(ga + gb, g0, rtol=1e-12, atol=1e-12 * np.abs(g0).max())


def test_nll_minimum_near_truth_on_large_sample(oracle):
    """On 2e5 events from the generative recipe, the 1D gradient at the truth is
    statistically compatible with zero (|g_j| / sqrt(sum terms^2) < 5)."""
    m = oracle.Model("1d", 0.3, 15.0)
    ev = {"t": synth.events_1d(200000, seed=9)}
    _, terms = oracle.nll_grad_terms(m, ev, TH1)
    g = terms.sum(axis=1)
    sd = np.sqrt((terms ** 2).sum(axis=1))
    assert np.all(np.abs(g[[0, 3]]) < 5 * sd[[0, 3]])


def test_fsum_is_exact_rounding():
    rng = np.random.default_rng(0)
    x = rng.normal(0, 1, 5000) * 10.0 ** rng.integers(-8, 8, 5000)
    exact = sum((Fraction(float(v)) for v in x), Fraction(0))
    assert math.fsum(x) == float(exact)
