"""GPU binned workloads (ipa_binned_generate, ipa_binned_smear, ipa_cls)
against the oracle (oracle/binned.py).

* Poisson counts bit-exact for means from 1e-9 to 3000 (pieces above 400),
  both hypotheses, a toy offset;
* smearing within 1e-15 of the histogram's maximum (different summation
  orders), edges included;
* CLs: the toy counts and CL values equal the oracle's exactly and every X
  within 1e-12 relative on a 2000-bin search; on the paper's configuration
  (10 000 bins on [5179, 5379], 10 000 toys) sampled toys' X against the
  oracle; a one-bin counting experiment against the closed form.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from oracle import binned
    from paper_1706_01420_gb300 import api
    return binned, G, torch, api


def _search(n_bins, lo=5179.0, hi=5379.0, m0=5279.6, s_sig=5.0, ns=70.0, nb=5000.0):
    """Signal: a Gaussian peak (shape before smearing) and the exponential
    background exp(-k m) with k = -0.001, both normalised to unit sum."""
    width = (hi - lo) / n_bins
    c = lo + (np.arange(n_bins) + 0.5) * width
    sig = np.exp(-0.5 * ((c - m0) / s_sig) ** 2)
    bkg = np.exp(0.001 * c)
    return width, sig / sig.sum() * ns, bkg / bkg.sum() * nb


def test_poisson_counts_bit_exact(env):
    B, G, torch, api = env
    lam = np.array([0.0, 1e-9, 0.2, 0.7, 1.5, 12.0, 37.5, 399.9, 400.0, 401.0, 950.0, 3000.0, -1.0] * 40)
    dl = torch.tensor(lam, device="cuda")
    for hyp, toy0, n_toys in ((0, 0, 3), (1, 5, 2), (0, 123456, 1)):
        got = api.ipa_binned_generate(dl, seed=2024, n_toys=n_toys, toy0=toy0, hypothesis=hyp).cpu().numpy()
        for k in range(n_toys):
            ref = B.generate_binned_fast(lam, 2024, toy0 + k, hyp)
            assert np.array_equal(got[k], ref), (hyp, toy0 + k)


def test_smearing_matches_oracle(env):
    B, G, torch, api = env
    rng = np.random.default_rng(3)
    h = rng.exponential(1.0, 3000)
    h[:40] = 0.0
    h[1500] = 50.0
    for width, sigma in ((0.02, 2.0), (0.5, 0.4), (1.0, 3.0)):
        got = api.ipa_binned_smear(torch.tensor(h, device="cuda"), width, sigma).cpu().numpy()
        ref = B.smear(h, width, sigma)
        assert np.max(np.abs(got - ref)) <= 1e-15 * h.max() * 4, (width, sigma)


def test_cls_matches_oracle(env):
    B, G, torch, api = env
    width, s, b = _search(2000)
    S = B.smear(s, width, 8.0)
    data = B.generate_binned_fast(S + b, 77, 0, 1)
    n_toys = 2000
    ref_cl, ref_n, (xb, xsb, xo) = B.cls(S, b, data, n_toys, seed=5)
    r = api.ipa_cls(torch.tensor(S, device="cuda"), torch.tensor(b, device="cuda"),
                    torch.tensor(data.astype(np.int32), device="cuda"), n_toys, 5, with_x=True)
    assert tuple(r["counts"].cpu().numpy()) == ref_n
    assert float(r["cl_b"]) == ref_cl[0] and float(r["cl_sb"]) == ref_cl[1] and float(r["cl_s"]) == ref_cl[2]
    np.testing.assert_allclose(r["x_b"].cpu().numpy(), xb, rtol=1e-12)
    np.testing.assert_allclose(r["x_sb"].cpu().numpy(), xsb, rtol=1e-12)
    assert float(r["x_obs"]) == pytest.approx(xo, rel=1e-12)
    assert 0 < ref_n[0] < n_toys and 0 < ref_n[1] < n_toys       # a non-trivial test


def test_cls_paper_configuration_sampled(env):
    """10 000 bins on [5179, 5379], 10 000 toys per hypothesis, ns = 70."""
    B, G, torch, api = env
    width, s, b = _search(10000)
    S_dev = api.ipa_binned_smear(torch.tensor(s, device="cuda"), width, 8.0)
    S_ref = B.smear(s, width, 8.0)
    np.testing.assert_allclose(S_dev.cpu().numpy(), S_ref, rtol=0, atol=1e-15 * s.max() * 4)
    data = B.generate_binned_fast(S_ref + b, 78, 0, 1)
    r = api.ipa_cls(torch.tensor(S_ref, device="cuda"), torch.tensor(b, device="cuda"),
                    torch.tensor(data.astype(np.int32), device="cuda"), 10000, 9, with_x=True)
    w = B.weights(S_ref, b)
    for k in (0, 4999, 9999):
        xb = B.statistic(B.generate_binned_fast(b, 9, k, 0), w)
        xsb = B.statistic(B.generate_binned_fast(S_ref + b, 9, k, 1), w)
        assert float(r["x_b"][k]) == pytest.approx(xb, rel=1e-12)
        assert float(r["x_sb"][k]) == pytest.approx(xsb, rel=1e-12)
    assert float(r["x_obs"]) == pytest.approx(B.statistic(data, w), rel=1e-12)
    nb, nsb = (int(v) for v in r["counts"].cpu())
    assert float(r["cl_s"]) == pytest.approx((nsb / 1e4) / (nb / 1e4))


def test_cls_counting_experiment_closed_form(env):
    from scipy import stats
    B, G, torch, api = env
    n_toys = 100000
    r = api.ipa_cls(torch.tensor([3.0], dtype=torch.float64, device="cuda"),
                    torch.tensor([5.0], dtype=torch.float64, device="cuda"),
                    torch.tensor([6], dtype=torch.int32, device="cuda"), n_toys, 13)
    for got, ref in ((float(r["cl_b"]), stats.poisson.cdf(6, 5.0)), (float(r["cl_sb"]), stats.poisson.cdf(6, 8.0))):
        assert abs(got - ref) < 5 * math.sqrt(ref * (1 - ref) / n_toys), (got, ref)
