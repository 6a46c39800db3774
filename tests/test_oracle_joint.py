"""Pins of the oracle's simultaneous fit over categories (oracle/joint.py).

* One category with the identity map is the model's own NLL and gradient.
* Categories that share every parameter are one fit of the concatenated events
  (NLL, gradient and the fitted minimum).
* Categories that share nothing are independent fits: the joint minimum is the
  separate minima side by side.
* The gradient, with parameters tied within a category and per-category
  constants, equals fourth-order central differences of the joint NLL.
"""
import numpy as np
import pytest

TH1 = np.array([0.66, 0.045, 0.0, 0.1])


@pytest.fixture(scope="module")
def J():
    from oracle import joint
    return joint


def _toys_1d(oracle, k, n, seed):
    m = oracle.Model("1d", 0.0, 15.0)
    evs = oracle.toygen(m, TH1, seed, [n] * k, [n // 9] * k)
    return m, [{"t": e["t"]} for e in evs]


def test_one_category_is_the_model(oracle, J):
    m, cats = _toys_1d(oracle, 1, 3000, 5)
    f0, g0 = oracle.nll_grad(m, cats[0], TH1)
    f, g = J.nll_grad(m, cats, [[0, 1, 2, 3]], None, TH1)
    assert f == f0
    np.testing.assert_array_equal(g, g0)


def test_all_shared_is_one_fit_of_the_union(oracle, J):
    m, cats = _toys_1d(oracle, 3, 2000, 6)
    union = {"t": np.concatenate([c["t"] for c in cats])}
    jmap = [[0, 1, 2, 3]] * 3
    th = TH1 * 1.02
    f, g = J.nll_grad(m, cats, jmap, None, th)
    f0, g0 = oracle.nll_grad(m, union, th)
    assert f == pytest.approx(f0, rel=1e-14)
    np.testing.assert_allclose(g, g0, rtol=1e-12, atol=1e-9)
    free = [0, 3]
    lo, hi = [0.1, 0.01, -1, 0.0], [3.0, 0.2, 1, 1.0]
    r = J.fit(m, cats, jmap, None, TH1, free, lo=lo, hi=hi)
    r0 = oracle.fit(m, union, TH1, free, lo=lo, hi=hi)
    assert r.status == r0.status == "CONVERGED"
    for j in free:
        assert abs(r.theta[j] - r0.theta[j]) < 1e-6 * r0.err[j]
        assert r.err[j] == pytest.approx(r0.err[j], rel=1e-5)


def test_nothing_shared_is_independent_fits(oracle, J):
    """Two categories, Gamma and f_b per category (joint 0, 1 and 2, 3), sigma
    and mu constants: the joint minimum is the two separate minima."""
    m, cats = _toys_1d(oracle, 2, 3000, 7)
    jmap = [[0, -1, -1, 1], [2, -1, -1, 3]]
    value = [[0.0, 0.045, 0.0, 0.0], [0.0, 0.045, 0.0, 0.0]]
    start = np.array([0.7, 0.12, 0.6, 0.08])
    lo, hi = [0.1, 0.0, 0.1, 0.0], [3.0, 1.0, 3.0, 1.0]
    r = J.fit(m, cats, jmap, value, start, [0, 1, 2, 3], lo=lo, hi=hi)
    assert r.status == "CONVERGED"
    for c in range(2):
        th0 = np.array([start[2 * c], 0.045, 0.0, start[2 * c + 1]])
        rc = oracle.fit(m, cats[c], th0, [0, 3], lo=[0.1, 0.01, -1, 0.0], hi=[3.0, 0.2, 1, 1.0])
        assert rc.status == "CONVERGED"
        for a, p in ((2 * c, 0), (2 * c + 1, 3)):
            assert abs(r.theta[a] - rc.theta[p]) < 1e-6 * rc.err[p]
            assert r.err[a] == pytest.approx(rc.err[p], rel=1e-5)


def test_gradient_matches_finite_differences(oracle, J):
    """4D model, three weighted categories: Gamma, sigma and the P-wave
    amplitudes shared, F_S and delta_S per category, mu and f_b per-category
    constants, except that f_b of category 2 is tied to sigma's joint
    parameter (one joint parameter feeding two model parameters of a
    category)."""
    m = oracle.Model("4d", 0.0, 15.0)
    rng = np.random.default_rng(3)
    cats = []
    for c in range(3):
        n = 800 + 300 * c
        cats.append({"t": np.minimum(rng.exponential(1.5, n), 14.9), "ck": rng.uniform(-1, 1, n),
                     "cl": rng.uniform(-1, 1, n), "phi": rng.uniform(-np.pi, np.pi, n),
                     "w": rng.normal(1.0, 0.2, n)})
    # joint: 0 Gamma, 1 sigma, 2 A0sq, 3 Apesq, 4 dpa, 5 dpe, 6..8 F_S per category, 9..11 dS per category
    jmap = []
    value = []
    for c in range(3):
        row = [0, 1, -1, -1, 2, 3, 4, 5, 6 + c, 9 + c]
        val = [0.0, 0.0, 0.01 * c, 0.1 + 0.05 * c, 0, 0, 0, 0, 0, 0]
        if c == 2:
            row[3] = 1          # f_b of category 2 tied to sigma's joint parameter
        jmap.append(row)
        value.append(val)
    th = np.array([0.66, 0.05, 0.52, 0.25, 3.2, 3.1, 0.04, 0.08, 0.12, 0.3, -0.5, 1.1])
    f, g = J.nll_grad(m, cats, jmap, value, th)

    def fj(j, d):
        tt = th.copy()
        tt[j] += d
        return J.nll(m, cats, jmap, value, tt)

    for j in range(th.size):
        h = 1e-5 * max(abs(th[j]), 0.1)
        fd = (8 * (fj(j, h) - fj(j, -h)) - (fj(j, 2 * h) - fj(j, -2 * h))) / (12 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(abs(g[j]), 1.0), (j, fd, g[j])
