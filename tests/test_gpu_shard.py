"""GPU checks of the event-sharded likelihood and of the stepwise fitter.

Ranks are emulated one after another in this process (no collective, no
kernel waits on another): each emulated rank runs ipa_nll_grad_shard on its
events, the group partials are concatenated in rank order, and
ipa_nll_grad_combine turns them into the NLL and gradient.  The result must be
bitwise ipa_nll_grad over all events (the sum over events of Sec. 3, with the
kernel's fixed reduction order), for every model, weighted or not, with the
cached angular basis, for 1 to 5 ranks, with empty ranks; and equal to the
oracle within the tolerances of the other parity tests.

The stepwise fitter (ipa_fit_begin / ipa_fit_advance / ipa_fit_end) driven by
ipa_nll_grad_segmented reproduces ipa_fit_batch bit for bit; driven by the
sharded NLL it gives the same fit; and a copy of its state taken between two
passes resumes the fit bit for bit.
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
TH1 = np.array([0.66, 0.045, 0.0, 0.1])
THT = np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.8, 0.3])
THP = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.8, 0.3, 0.8, 0.0])
LO4 = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
HI4 = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2])
STEP4 = np.array([0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api, shard
    return oracle, G, torch, api, shard


def _sharded(torch, api, shard, m, ev, theta, world, cached=False):
    n = int(ev["t"].numel())
    blocks = []
    for r in range(world):
        lo, hi = shard.shard_bounds(n, r, world)
        local = {k: v[lo:hi] for k, v in ev.items() if k != "fk"}
        if cached:
            local["fk"] = api.ipa_angular_basis(m, local)
        _, groups = api.ipa_nll_grad_shard(m, local, theta)
        blocks.append(groups)
    allg = torch.cat(blocks) if blocks else torch.empty(0, api.ipa_shard_width(m), dtype=torch.float64,
                                                        device="cuda")
    return api.ipa_nll_grad_combine(m, theta, allg, cached).cpu().numpy()


CASES = {
    "4d": lambda api: (api.model_4d(0.0, 15.0), synth.events_4d(100_003, 61), TH4),
    "4d_weighted": lambda api: (api.model_4d(0.0, 15.0), synth.events_4d(70_001, 62, weighted=True), TH4),
    "1d": lambda api: (api.model_1d(0.3, 15.0), {"t": synth.events_1d(90_000, 63)}, TH1),
    "tagged": lambda api: (api.model_tagged(0.0, 15.0), synth.events_tagged(50_000, 64, weighted=True), THT),
    "phis": lambda api: (api.model_phis(0.0, 15.0), synth.events_phis(40_000, 65), THP),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_equals_one_gpu_bitwise(env, case):
    O, G, torch, api, shard = env
    m, cols, th = CASES[case](api)
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    one = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
    for world in (1, 2, 3, 5):
        got = _sharded(torch, api, shard, m, ev, theta, world)
        assert np.array_equal(got, one), (case, world, got - one)
    if case in ("4d", "4d_weighted", "1d"):
        m_o = O.Model(case[:2], m.t_lo, m.t_hi)
        f_ref, g_ref = O.nll_grad(m_o, cols, th)
        logl, _ = O.nll_grad_terms(m_o, cols, th)
        G.assert_nll_grad_close(one, f_ref, g_ref, G.grad_scale(O, m_o, cols, th), math.fsum(np.abs(logl)))


@pytest.mark.parametrize("kind", ["4d", "phis"])
def test_sharded_cached_basis_bitwise(env, kind):
    O, G, torch, api, shard = env
    if kind == "4d":
        m, cols, th = api.model_4d(0.0, 15.0), synth.events_4d(60_000, 66), TH4
    else:
        m, cols, th = api.model_phis(0.0, 15.0), synth.events_phis(40_000, 67), THP
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    one = api.ipa_nll_grad(m, dict(ev, fk=api.ipa_angular_basis(m, ev)), theta).cpu().numpy()
    for world in (2, 3):
        assert np.array_equal(_sharded(torch, api, shard, m, ev, theta, world, cached=True), one)


def test_shards_with_empty_ranks_and_empty_input(env):
    O, G, torch, api, shard = env
    m = api.model_4d(0.0, 15.0)
    cols = synth.events_4d(20_000, 68)          # two groups: with 5 ranks three are empty
    ev = G.to_dev(cols)
    theta = torch.tensor(TH4, device="cuda")
    one = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
    assert [shard.shard_bounds(20_000, r, 5)[1] - shard.shard_bounds(20_000, r, 5)[0] for r in range(5)].count(0) == 3
    assert np.array_equal(_sharded(torch, api, shard, m, ev, theta, 5), one)
    empty = {k: v[:0] for k, v in ev.items()}
    assert np.array_equal(_sharded(torch, api, shard, m, empty, theta, 2), np.zeros(11))


def _stepwise(torch, api, m, params, theta0, evaluate, max_iter=200, tol=1e-9, stop_after=None, state=None):
    n_fits, P = theta0.shape
    if state is None:
        state = api.fit_state_new(n_fits, P, "cuda")
        api.ipa_fit_begin(m, params, theta0, state, max_iter=max_iter, tol=tol)
    points = api.fit_state_points(state, n_fits, P)
    res = torch.empty(n_fits, 1 + P, dtype=torch.float64, device="cuda")
    n_active = torch.ones(1, dtype=torch.int32, device="cuda")
    passes = 0
    while True:
        evaluate(points, res)
        api.ipa_fit_advance(m, n_fits, res, state, n_active)
        passes += 1
        if stop_after is not None and passes == stop_after:
            return state
        if int(n_active.item()) == 0:
            break
        assert passes < 2000
    return api.ipa_fit_end(m, n_fits, state)


def _toys(O, api, n_toys, per, seed):
    m_o = O.Model("4d", 0.0, 15.0)
    n_sig, n_bkg = synth.toy_sizes(n_toys, per, TH4[3], seed=seed)
    toys = [O.toy_one(m_o, TH4, seed, k, int(n_sig[k]), int(n_bkg[k])) for k in range(n_toys)]
    sizes = [t["t"].size for t in toys]
    cols = {k: np.concatenate([t[k] for t in toys]) for k in toys[0]}
    return cols, np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _params(api, th):
    return [api.Param(float(th[i]), float(LO4[i]), float(HI4[i]), float(STEP4[i])) for i in range(10)]


def test_stepwise_fit_equals_fit_batch_and_resumes_from_a_copy(env):
    O, G, torch, api, shard = env
    cols, off = _toys(O, api, 4, 6000, 71)
    ev = G.to_dev(cols)
    m = api.model_4d(0.0, 15.0)
    off_d = torch.tensor(off, device="cuda")
    params = _params(api, TH4)
    start = np.tile(TH4, (4, 1))
    start[:, 0] += 0.02
    batch = api.ipa_fit_batch(m, ev, off_d, params, torch.tensor(start, device="cuda"), max_iter=200, tol=1e-9)

    def evaluate(points, res):
        api.ipa_nll_grad_segmented(m, ev, off_d, points, res)

    step = _stepwise(torch, api, m, params, torch.tensor(start, device="cuda"), evaluate)
    for key in ("theta", "err", "nll", "status", "iters", "passes"):
        assert np.array_equal(step[key].cpu().numpy(), batch[key].cpu().numpy()), key
    # a copy of the state after 11 passes, restored into a fresh buffer, resumes bitwise
    state = _stepwise(torch, api, m, params, torch.tensor(start, device="cuda"), evaluate, stop_after=11)
    saved = state.cpu().numpy().copy()
    first = _stepwise(torch, api, m, params, torch.tensor(start, device="cuda"), evaluate, state=state)
    restored = torch.tensor(saved, device="cuda")
    second = _stepwise(torch, api, m, params, torch.tensor(start, device="cuda"), evaluate, state=restored)
    for key in ("theta", "err", "nll", "status", "iters", "passes"):
        assert np.array_equal(first[key].cpu().numpy(), second[key].cpu().numpy()), key
        assert np.array_equal(first[key].cpu().numpy(), batch[key].cpu().numpy()), key


def test_sharded_fit_equals_one_gpu_fit(env):
    """One fit of 1.2e5 events whose NLL and gradient come from 3 emulated ranks
    each pass: the same fit, bit for bit, as ipa_fit_batch on one GPU."""
    O, G, torch, api, shard = env
    cols, off = _toys(O, api, 1, 120_000, 72)
    ev = G.to_dev(cols)
    m = api.model_4d(0.0, 15.0)
    params = _params(api, TH4)
    start = TH4.copy()
    start[[0, 4, 6]] += [0.02, 0.01, 0.05]
    off_d = torch.tensor(off, device="cuda")
    batch = api.ipa_fit_batch(m, ev, off_d, params, torch.tensor(start[None, :], device="cuda"), max_iter=200,
                              tol=1e-9)

    def evaluate(points, res):
        res[0] = torch.tensor(_sharded(torch, api, shard, m, ev, points[0], 3), device="cuda")

    step = _stepwise(torch, api, m, params, torch.tensor(start[None, :], device="cuda"), evaluate)
    assert int(step["status"][0]) == 0
    for key in ("theta", "err", "nll", "status", "iters", "passes"):
        assert np.array_equal(step[key].cpu().numpy(), batch[key].cpu().numpy()), key
