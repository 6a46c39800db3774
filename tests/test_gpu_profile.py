"""GPU HESSE (ipa_hesse) and MINOS (ipa_minos) against the oracle
(oracle/profile.py).

* covariance, correlations and errors within 1e-3 (relative to
  sqrt(C_ii C_jj); the bar of the fitted errors) of the oracle's at the same
  point, for the 1D, 4D and tagged models; a fit in a batch gives bitwise its
  solo result;
* MINOS interval ends within 1e-5 sigma of the oracle's, with one free
  parameter (the NLL crossing), with nuisance parameters profiled out, and at
  a parameter limit (status IPA_MINOS_AT_LIMIT); batch = solo bitwise.
"""
import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH1 = np.array([0.66, 0.045, 0.0, 0.1])
LO1, HI1 = np.array([0.1, 0.01, -1.0, 0.0]), np.array([3.0, 0.2, 1.0, 1.0])
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
LO4 = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
HI4 = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2])
TAG = np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.8, 0.3])
LOT = np.array([0.3, 0.01, -0.1, 0.0, -0.5, 10.0, -3.1, 0.0])
HIT = np.array([1.5, 0.2, 0.1, 0.5, 0.5, 25.0, 3.1, 0.5])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from oracle import profile
    from paper_1706_01420_gb300 import api
    return oracle, profile, G, torch, api


def _params(api, th, lo, hi, free):
    return [api.Param(float(th[i]), float(lo[i]), float(hi[i]), float(hi[i] - lo[i]) / 50, fixed=i not in free)
            for i in range(len(th))]


def _cols_dev(G, torch, parts):
    cols = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    off = torch.tensor(np.concatenate([[0], np.cumsum([p["t"].size for p in parts])]), dtype=torch.int64,
                       device="cuda")
    return G.to_dev(cols), off


def _assert_cov_close(C, Cref, free, rtol=1e-4):
    d = np.sqrt(np.diag(Cref))
    for a in free:
        for b in free:
            assert abs(C[a, b] - Cref[a, b]) <= rtol * d[a] * d[b], (a, b, C[a, b], Cref[a, b])


@pytest.mark.parametrize("kind", ["1d", "4d", "tag"])
def test_hesse_matches_oracle(env, kind):
    O, P, G, torch, api = env
    if kind == "1d":
        m_o, m = O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0)
        cols, th, lo, hi, free = {"t": synth.events_1d(50000, 1)}, TH1 + [0.01, 0, 0, -0.01], LO1, HI1, [0, 3]
    elif kind == "4d":
        m_o, m = O.Model("4d", 0.0, 15.0), api.model_4d(0.0, 15.0)
        cols = O.toy_one(m_o, TH4, 2, 0, 18000, 2000)
        th, lo, hi, free = TH4, LO4, HI4, list(range(10))
    else:
        # Gamma, f_b, Dm, phi_s (with DG free as well, Gamma, DG and phi_s are
        # correlated to |rho| > 0.99 at this size and the covariance depends on
        # the finite-difference steps more than on anything else)
        m_o, m = O.Model("tag", 0.0, 15.0), api.model_tagged(0.0, 15.0)
        cols = O.toy_one(m_o, TAG, 3, 0, 18000, 2000)
        th, lo, hi, free = TAG, LOT, HIT, [0, 3, 5, 6]
    Cref, eref, corr_ref, _ = P.hesse(m_o, cols, th, free)
    ev, off = _cols_dev(G, torch, [cols])
    r = api.ipa_hesse(m, ev, off, _params(api, th, lo, hi, free), torch.tensor(th[None, :], device="cuda"))
    C = r["cov"].cpu().numpy()[0]
    assert int(r["status"][0]) == 0
    # both sides take finite differences of the analytic gradient, with
    # different steps: the bar is that of the fitted errors, 1e-3
    _assert_cov_close(C, Cref, free, rtol=1e-3)
    np.testing.assert_allclose(r["err"].cpu().numpy()[0][free], eref[free], rtol=1e-3)
    corr = r["corr"].cpu().numpy()[0][np.ix_(free, free)]
    np.testing.assert_allclose(corr, corr_ref, atol=1e-3)
    fixed = [p for p in range(len(th)) if p not in free]
    assert np.all(C[fixed, :] == 0) and np.all(C[:, fixed] == 0)


def test_hesse_batch_equals_solo(env):
    O, P, G, torch, api = env
    m = api.model_4d(0.0, 15.0)
    parts = [synth.events_4d(n, 30 + n) for n in (3000, 700, 5000)]
    ev, off = _cols_dev(G, torch, parts)
    params = _params(api, TH4, LO4, HI4, list(range(10)))
    ths = np.stack([TH4, TH4 * 1.01, TH4 * 0.99])
    batch = api.ipa_hesse(m, ev, off, params, torch.tensor(ths, device="cuda"))
    for k in (0, 2):
        e1, o1 = _cols_dev(G, torch, [parts[k]])
        solo = api.ipa_hesse(m, e1, o1, params, torch.tensor(ths[k:k + 1], device="cuda"))
        for key in ("cov", "corr", "err", "status"):
            assert torch.equal(solo[key][0], batch[key][k]), (k, key)


def _minos_case(env, m_o, m, cols, th0, lo, hi, free, scan, tol_fit=1e-12):
    """Oracle fit -> minimum; GPU HESSE and MINOS at the oracle's minimum; oracle MINOS."""
    O, P, G, torch, api = env
    r = O.fit(m_o, cols, th0, free, lo=lo, hi=hi, tol=tol_fit)
    ev, off = _cols_dev(G, torch, [cols])
    params = _params(api, r.theta, lo, hi, free)
    th = torch.tensor(r.theta[None, :], device="cuda")
    hs = api.ipa_hesse(m, ev, off, params, th)
    nll = api.ipa_nll(m, ev, th[0])
    got = api.ipa_minos(m, ev, off, params, th, nll, hs["cov"], scan)
    C, err, _, _ = P.hesse(m_o, cols, r.theta, free)
    ref = {j: P.minos(m_o, cols, r.theta, r.nll, free, j, err[j], lo=lo, hi=hi) for j in scan}
    return r, err, {k: v.cpu().numpy()[0] for k, v in got.items()}, ref


def test_minos_single_free_parameter(env):
    O, P, G, torch, api = env
    cols = {"t": synth.events_1d(5000, 11)}
    r, err, got, ref = _minos_case(env, O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0), cols, TH1, LO1, HI1,
                                   [0], [0])
    (elo, ehi), st = ref[0]
    assert st == ("OK", "OK") and tuple(got["status"][0]) == (0, 0)
    assert abs(got["lo"][0] - elo) < 1e-5 * err[0] and abs(got["hi"][0] - ehi) < 1e-5 * err[0]


def test_minos_profiles_out_nuisance_parameters(env):
    O, P, G, torch, api = env
    cols = {"t": synth.events_1d(20000, 12)}
    r, err, got, ref = _minos_case(env, O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0), cols, TH1, LO1, HI1,
                                   [0, 3], [0, 3])
    for j in (0, 3):
        (elo, ehi), st = ref[j]
        assert st == ("OK", "OK") and tuple(got["status"][j]) == (0, 0), (j, got["status"][j])
        assert abs(got["lo"][j] - elo) < 1e-5 * err[j], (j, got["lo"][j], elo)
        assert abs(got["hi"][j] - ehi) < 1e-5 * err[j], (j, got["hi"][j], ehi)
    assert got["lo"][1] == 0 and tuple(got["status"][1]) == (5, 5)   # sigma: fixed, not scanned


def test_minos_tagged_model(env):
    O, P, G, torch, api = env
    m_o = O.Model("tag", 0.0, 15.0)
    cols = O.toy_one(m_o, TAG, 6, 0, 9000, 1000)
    free = [0, 3, 4, 5, 6]
    r, err, got, ref = _minos_case(env, m_o, api.model_tagged(0.0, 15.0), cols, TAG, LOT, HIT, free, [6],
                                   tol_fit=1e-10)
    (elo, ehi), st = ref[6]
    assert st == ("OK", "OK") and tuple(got["status"][6]) == (0, 0)
    assert abs(got["lo"][6] - elo) < 1e-5 * err[6] and abs(got["hi"][6] - ehi) < 1e-5 * err[6]


def test_minos_at_a_limit(env):
    """No background in the sample: the lower interval of f_b runs into f_b = 0."""
    O, P, G, torch, api = env
    truth = {"Gamma": 0.66, "sigma": 0.045, "mu": 0.0, "f_b": 0.0}
    cols = {"t": synth.events_1d(2000, 10, truth=truth)}
    r, err, got, ref = _minos_case(env, O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0), cols,
                                   np.array([0.66, 0.045, 0.0, 0.02]), LO1, HI1, [0, 3], [3], tol_fit=1e-10)
    (elo, ehi), st = ref[3]
    assert st == ("LIMIT", "OK")
    assert int(got["status"][3][0]) == 2 and got["lo"][3] == -r.theta[3]
    assert int(got["status"][3][1]) == 0 and abs(got["hi"][3] - ehi) < 1e-5 * err[3]


def test_minos_batch_equals_solo(env):
    O, P, G, torch, api = env
    m = api.model_1d(0.3, 15.0)
    parts = [{"t": synth.events_1d(n, 40 + n)} for n in (4000, 9000, 2500)]
    ev, off = _cols_dev(G, torch, parts)
    params = _params(api, TH1, LO1, HI1, [0, 3])
    th = torch.tensor(np.tile(TH1, (3, 1)), device="cuda")
    fit = api.ipa_fit_batch(m, ev, off, params, th.clone(), tol=1e-10)
    hs = api.ipa_hesse(m, ev, off, params, fit["theta"])
    batch = api.ipa_minos(m, ev, off, params, fit["theta"], fit["nll"], hs["cov"], [0, 3])
    for k in (0, 2):
        e1, o1 = _cols_dev(G, torch, [parts[k]])
        f1 = api.ipa_fit_batch(m, e1, o1, params, th[:1].clone(), tol=1e-10)
        h1 = api.ipa_hesse(m, e1, o1, params, f1["theta"])
        solo = api.ipa_minos(m, e1, o1, params, f1["theta"], f1["nll"], h1["cov"], [0, 3])
        for key in ("lo", "hi", "status"):
            assert torch.equal(solo[key][0], batch[key][k]), (k, key)
        assert torch.all(batch["status"][k][[0, 3]] == 0)
