"""Cached angular basis (ipa_angular_basis): the basis equals the oracle's f_k,
and likelihood, segmented and fit calls that read it agree with the oracle."""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


@pytest.mark.parametrize("n", [1, 2, 511, 100001])
def test_basis_matches_oracle(env, n):
    O, G, torch, api = env
    cols = synth.events_4d(n, n)
    ev = G.to_dev(cols)
    fk = api.ipa_angular_basis(api.model_4d(), ev).cpu().numpy()
    ref = O.angular_basis(cols["ck"], cols["cl"], cols["phi"])
    # absolute: sin(theta) = sqrt(1 - cos^2) is ill-conditioned near |cos| = 1, where the
    # two sides round 1 - cos^2 differently (the GPU forms it with one FMA)
    np.testing.assert_allclose(fk[:, :n], ref, rtol=0, atol=4e-15)


@pytest.mark.parametrize("n", [0, 513, 1_000_000])
def test_nll_grad_with_basis_matches_oracle(env, n):
    O, G, torch, api = env
    cols = synth.events_4d(n, 7, weighted=True)
    ev = G.to_dev(cols)
    m = api.model_4d()
    if n:
        ev["fk"] = api.ipa_angular_basis(m, ev)
    got = api.ipa_nll_grad(m, ev, torch.tensor(TH4, device="cuda")).cpu().numpy()
    if n == 0:
        assert np.all(got == 0)
        return
    mo = O.Model("4d", 0.0, 15.0)
    f_ref, g_ref = O.nll_grad(mo, cols, TH4)
    logl, _ = O.nll_grad_terms(mo, cols, TH4)
    G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, mo, cols, TH4), math.fsum(np.abs(logl)))


def test_unweighted_full_size_and_a_nan_in_the_basis(env):
    """Whole tiles read the cached basis on the fixed-point path (the f_k in
    Q62): unweighted, 1e6 events, against the oracle; and one event whose
    cached f_k is NaN makes the NLL and the gradient NaN, as the FP64 loop
    does (the tile falls back to it)."""
    O, G, torch, api = env
    cols = synth.events_4d(1_000_000, 8)
    ev = G.to_dev(cols)
    m = api.model_4d()
    ev["fk"] = api.ipa_angular_basis(m, ev)
    theta = torch.tensor(TH4, device="cuda")
    got = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
    mo = O.Model("4d", 0.0, 15.0)
    f_ref, g_ref = O.nll_grad(mo, cols, TH4)
    logl, _ = O.nll_grad_terms(mo, cols, TH4)
    G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, mo, cols, TH4), math.fsum(np.abs(logl)))
    fk = ev["fk"].clone()
    fk[3, 4321] = float("nan")
    bad = api.ipa_nll_grad(m, dict(ev, fk=fk), theta).cpu().numpy()
    assert np.isnan(bad[0]) and np.isnan(bad[1:]).any()


def test_fit_with_basis_matches_oracle(env):
    O, G, torch, api = env
    mo = O.Model("4d", 0.0, 15.0)
    toy = O.toy_one(mo, TH4, 21, 3, 18000, 2000)
    ev = G.to_dev(toy)
    m = api.model_4d()
    ev["fk"] = api.ipa_angular_basis(m, ev)
    lo = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
    hi = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2])
    step = np.array([0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2])
    params = [api.Param(float(TH4[i]), float(lo[i]), float(hi[i]), float(step[i])) for i in range(10)]
    off = torch.tensor([0, 20000], dtype=torch.int64, device="cuda")
    r = api.ipa_fit_batch(m, ev, off, params, torch.tensor(TH4[None, :], device="cuda"), tol=1e-9)
    ref = O.fit(mo, toy, TH4, list(range(10)), lo, hi, tol=1e-10)
    assert int(r["status"][0]) == 0 and ref.status == "CONVERGED"
    np.testing.assert_array_less(np.abs(r["theta"][0].cpu().numpy() - ref.theta), 1e-6 * ref.err)
