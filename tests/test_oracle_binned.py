"""Pins of the oracle's binned workloads (oracle/binned.py).

* the Poisson sampler is the inversion of the exact CDF (scipy's) for
  uniforms away from the CDF steps, its counts follow the Poisson pmf (chi^2)
  for means from 0.3 to 3000 (including the split above 400), and the
  vectorised generator equals the bin-by-bin one;
* smearing a Gaussian histogram by a Gaussian gives the Gaussian with the
  variances added, and keeps the total away from the edges;
* CLs of a one-bin counting experiment equals the closed form
  CL_s+b = F(n_obs; s + b), CL_b = F(n_obs; b) (Poisson CDFs) within the
  binomial error of the toys.
"""
import math

import numpy as np
import pytest
from scipy import stats


@pytest.fixture(scope="module")
def B():
    from oracle import binned
    return binned


def test_inversion_is_the_exact_cdf(B):
    rng = np.random.default_rng(0)
    for nu in (0.3, 4.0, 37.0, 399.0):
        for u in rng.uniform(0, 1, 400):
            n = B.poisson_piece(nu, float(u))
            lo = stats.poisson.cdf(n - 1, nu) if n else 0.0
            hi = stats.poisson.cdf(n, nu)
            if min(abs(u - lo), abs(u - hi)) < 1e-11:
                continue          # a CDF step within rounding
            assert lo < u <= hi, (nu, u, n, lo, hi)


@pytest.mark.parametrize("lam", [0.3, 4.0, 37.0, 950.0, 3000.0])
def test_counts_follow_the_poisson_pmf(B, lam):
    n_bins = 4000
    counts = B.generate_binned_fast(np.full(n_bins, lam), seed=7, toy=3)
    mean, var = counts.mean(), counts.var(ddof=1)
    assert abs(mean - lam) < 5 * math.sqrt(lam / n_bins)
    assert abs(var / lam - 1) < 5 * math.sqrt(2.0 / n_bins)
    # chi^2 over the central quantiles of the pmf
    lo, hi = int(stats.poisson.ppf(0.01, lam)), int(stats.poisson.ppf(0.99, lam))
    edges = np.unique(np.linspace(lo, hi + 1, 12).astype(int))
    obs = np.histogram(counts, edges)[0]
    exp = n_bins * np.diff(stats.poisson.cdf(edges - 1, lam))
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    dof = len(obs)
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_vectorised_generator_equals_the_plain_one(B):
    lam = np.array([0.0, 0.2, 1.5, 12.0, 399.9, 400.0, 401.0, 1234.5, 1e-9])
    for toy, hyp in ((0, 0), (5, 1), (12345, 0)):
        assert np.array_equal(B.generate_binned(lam, 99, toy, hyp), B.generate_binned_fast(lam, 99, toy, hyp))


def test_smearing_adds_variances(B):
    width, n = 0.02, 10000
    c = 5179.0 + (np.arange(n) + 0.5) * width
    s1, s0, m0 = 1.5, 2.0, 5279.0
    g = np.exp(-0.5 * ((c - m0) / s1) ** 2)
    out = B.smear(g, width, s0)
    st = math.hypot(s1, s0)
    ref = np.exp(-0.5 * ((c - m0) / st) ** 2) * (s1 / st)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)
    assert math.fsum(out) == pytest.approx(math.fsum(g), rel=1e-14)


def test_cls_of_a_counting_experiment(B):
    s, b, n_obs, n_toys = np.array([3.0]), np.array([5.0]), np.array([6]), 4000
    (cl_b, cl_sb, cl_s), (nb, nsb), _ = B.cls(s, b, n_obs, n_toys, seed=11)
    ref_b, ref_sb = stats.poisson.cdf(6, 5.0), stats.poisson.cdf(6, 8.0)
    for got, ref in ((cl_b, ref_b), (cl_sb, ref_sb)):
        assert abs(got - ref) < 5 * math.sqrt(ref * (1 - ref) / n_toys), (got, ref)
    assert cl_s == pytest.approx(cl_sb / cl_b)
