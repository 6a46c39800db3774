"""GPU batched fits (ipa_fit_batch) against the oracle's fits.

* fitted parameters within 1e-6 sigma of the oracle's minimum, NLL at the
  minimum to 1e-12, errors (sqrt diag of the inverse Hessian) to 1e-3;
* a fit packed in a batch is bitwise the same fit run alone;
* pulls of GPU-generated, GPU-fitted toys have mean 0 and width 1.
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH1 = np.array([0.66, 0.045, 0.0, 0.1])
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
LO4 = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
HI4 = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2])
STEP4 = np.array([0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def _params(api, th, lo, hi, step, free):
    return [api.Param(float(th[i]), float(lo[i]), float(hi[i]), float(step[i]), fixed=i not in free)
            for i in range(len(th))]


def _fit(env, m, toys, th0, params, tol=1e-9):
    O, G, torch, api = env
    sizes = [t["t"].size for t in toys]
    cols = {k: np.concatenate([t[k] for t in toys]) for k in toys[0]}
    ev = G.to_dev(cols)
    off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    theta = torch.tensor(np.tile(th0, (len(toys), 1)), device="cuda")
    r = api.ipa_fit_batch(m, ev, off, params, theta, max_iter=200, tol=tol)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def test_fit_1d_config1_matches_oracle(env):
    """1e5 events on [0.3, 15] ps; Gamma and f_b free.  sigma and mu are fixed: on
    this range the resolution leaves no trace in the data (identifiability)."""
    O, G, torch, api = env
    t = synth.events_1d(100_000, 0)
    free = [0, 3]
    lo, hi = np.array([0.3, 0.01, -0.1, 0.0]), np.array([1.5, 0.2, 0.1, 0.5])
    step = np.array([0.01, 0.003, 0.002, 0.005])
    start = TH1 + np.array([0.03, 0, 0, -0.02])
    r = _fit(env, api.model_1d(0.3, 15.0), [{"t": t}], start, _params(api, start, lo, hi, step, free))
    ref = O.fit(O.Model("1d", 0.3, 15.0), {"t": t}, start, free, lo, hi, tol=1e-10)
    assert r["status"][0] == 0 and ref.status == "CONVERGED"
    for j in free:
        assert abs(r["theta"][0, j] - ref.theta[j]) < 1e-6 * ref.err[j], j
        assert r["err"][0, j] == pytest.approx(ref.err[j], rel=1e-3)
    assert r["nll"][0] == pytest.approx(ref.nll, rel=1e-12)


def test_fit_4d_matches_oracle_and_batch_equals_solo(env):
    O, G, torch, api = env
    m_o = O.Model("4d", 0.0, 15.0)
    n_sig, n_bkg = synth.toy_sizes(6, 2e4, TH4[3], seed=1)
    toys = [O.toy_one(m_o, TH4, 5, k, int(n_sig[k]), int(n_bkg[k])) for k in range(6)]
    free = list(range(10))
    params = _params(api, TH4, LO4, HI4, STEP4, free)
    m = api.model_4d(0.0, 15.0)
    batch = _fit(env, m, toys, TH4, params)
    for k in (0, 3):
        solo = _fit(env, m, [toys[k]], TH4, params)
        for key in ("theta", "err", "nll", "status", "iters"):
            assert np.array_equal(solo[key][0], batch[key][k]), (k, key)
    for k in (0, 4):
        ref = O.fit(m_o, toys[k], TH4, free, LO4, HI4, tol=1e-10)
        assert ref.status == "CONVERGED"
        assert batch["status"][k] == 0
        np.testing.assert_array_less(np.abs(batch["theta"][k] - ref.theta), 1e-6 * ref.err)
        np.testing.assert_allclose(batch["err"][k], ref.err, rtol=1e-3)
        assert batch["nll"][k] == pytest.approx(ref.nll, rel=1e-12)


def test_fit_runs_as_one_device_loop_and_reuses_its_graph(env, tmp_path, monkeypatch):
    """With IPA_TRACE set, ipa_fit_batch reports that the minimisation ran as one
    graph launch with a device-side loop; consecutive fits of toys of the same
    event set give the same results as a fresh call."""
    O, G, torch, api = env
    trace = tmp_path / "trace.jsonl"
    monkeypatch.setenv("IPA_TRACE", str(trace))
    m_o = O.Model("4d", 0.0, 15.0)
    toys = [O.toy_one(m_o, TH4, 9, k, 4500, 500) for k in range(3)]
    cols = {k: np.concatenate([t[k] for t in toys]) for k in toys[0]}
    ev = G.to_dev(cols)
    m = api.model_4d(0.0, 15.0)
    params = _params(api, TH4, LO4, HI4, STEP4, list(range(10)))
    res = []
    for k in (0, 1, 2, 1):
        off = torch.tensor([5000 * k, 5000 * (k + 1)], dtype=torch.int64, device="cuda")
        r = api.ipa_fit_batch(m, ev, off, params, torch.tensor(TH4[None, :], device="cuda"), tol=1e-8)
        res.append(r["theta"][0].cpu().numpy())
    assert np.array_equal(res[1], res[3])
    import json
    lines = [json.loads(x) for x in trace.read_text().splitlines()]
    assert len(lines) == 4 and all(x["loop"] == "device" for x in lines)


def _toy_pulls(env, n_toys, mean_size, seed, gen_seed):
    """Pulls (theta - truth) / error of n_toys GPU-generated toys of
    Poisson(mean_size) events fitted in one batch, all ten parameters free,
    over the converged fits."""
    O, G, torch, api = env
    n_sig, n_bkg = synth.toy_sizes(n_toys, mean_size, TH4[3], seed=seed)
    sizes = n_sig + n_bkg
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(off[-1])
    dev = lambda a: torch.tensor(a, dtype=torch.int64, device="cuda")
    cols = {k: torch.empty(total, dtype=torch.float64, device="cuda") for k in ("t", "ck", "cl", "phi")}
    m = api.model_4d(0.0, 15.0)
    api.ipa_toygen(m, torch.tensor(TH4, device="cuda"), gen_seed, dev(n_sig), dev(n_bkg), dev(off[:-1]), cols)
    free = list(range(10))
    theta = torch.tensor(np.tile(TH4, (n_toys, 1)), device="cuda")
    r = api.ipa_fit_batch(m, cols, dev(off), _params(api, TH4, LO4, HI4, STEP4, free), theta,
                          max_iter=200, tol=1e-8)
    st = r["status"].cpu().numpy()
    th = r["theta"].cpu().numpy()
    er = r["err"].cpu().numpy()
    ok = st == 0
    assert ok.mean() > 0.95, np.bincount(st)
    del cols
    torch.cuda.empty_cache()
    pulls = (th[ok] - TH4) / er[ok]
    print(f"PULLS {n_toys} toys of Poisson({mean_size:g}): mean", np.round(pulls.mean(axis=0), 4).tolist(),
          "width", np.round(pulls.std(axis=0, ddof=1), 4).tolist())
    return pulls


@pytest.mark.slow
def test_gpu_toy_pulls_all_parameters_2e5(env):
    """256 toys of Poisson(2e5) events: the pulls of all ten parameters have
    mean 0 and width 1, |mean| < 3.5/sqrt(n) and |width - 1| < 3.5/sqrt(2n) +
    0.03 (the HESSE errors at NLL_min + 1/2 of Sec. 3 are the standard
    deviations of the estimates)."""
    pulls = _toy_pulls(env, 256, 2e5, seed=3, gen_seed=79)
    n = pulls.shape[0]
    for j in range(10):
        p = pulls[:, j]
        assert abs(p.mean()) < 3.5 / math.sqrt(n), (j, p.mean())
        assert abs(p.std(ddof=1) - 1) < 3.5 / math.sqrt(2 * n) + 0.03, (j, p.std(ddof=1))


@pytest.mark.slow
def test_gpu_toy_pulls(env):
    """256 GPU-generated toys of Poisson(2e4) events fitted in one batch: pulls of
    the eight parameters other than sigma and mu have mean 0 and width 1 within
    3.5 standard errors.  sigma and mu are measured only by the ~1e3 events of
    the turn-on at t ~ 0; at this size their pulls are biased (the maximum-
    likelihood bias of order 1/sqrt(N) in pull units: mu's mean pull is about
    +0.25 at 2e4 events (4096 toys) and 0.15 +- 0.06 at 2e5, where
    test_gpu_toy_pulls_all_parameters_2e5 checks all ten with the strict
    bound), so here they get a looser one."""
    pulls = _toy_pulls(env, 256, 2e4, seed=2, gen_seed=77)
    se = 1 / math.sqrt(pulls.shape[0])
    for j in (0, 3, 4, 5, 6, 7, 8, 9):
        p = pulls[:, j]
        assert abs(p.mean()) < 3.5 * se, (j, p.mean())
        assert abs(p.std(ddof=1) - 1) < 3.5 * se / math.sqrt(2) + 0.03, (j, p.std(ddof=1))
    for j in (1, 2):
        p = pulls[:, j]
        assert abs(p.mean()) < 0.5 and 0.8 < p.std(ddof=1) < 1.35, (j, p.mean(), p.std(ddof=1))
