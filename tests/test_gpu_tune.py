"""Launch geometry and its autotuner: no result depends on the geometry.

The likelihood kernel's summation order is fixed by 512-event tiles and
32-tile groups, so every block size, resident-warp count and tiles-per-take
choice must give the same NLL and gradient bit for bit, and a batched fit must
give the same fitted parameters before and after the autotuner changes the
geometry.  Parity of the values themselves with the oracle is covered by
test_gpu_nll.py; here one oracle check ties the geometry sweep to it.
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
GEOMETRIES = [{"warps_per_block": w, "warps_per_sm": s, "tiles_per_take": k}
              for w in (1, 2, 4, 8) for s in (0, 3, 64) for k in (1, 2, 4)]


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def _restore_default(api, m, n, n_seg=1, grad=True, cached=False):
    api.ipa_launch_config_set(m, n, {"warps_per_block": 1, "warps_per_sm": 0, "tiles_per_take": 1},
                              n_seg=n_seg, grad=grad, cached=cached)


@pytest.mark.parametrize("n", [1, 513, 16385, 70001])
def test_every_geometry_gives_the_same_bits(env, n):
    O, G, torch, api = env
    m = api.model_4d()
    cols = synth.events_4d(n, 40 + n, weighted=True)
    ev = G.to_dev(cols)
    theta = torch.tensor(TH4, device="cuda")
    ref = None
    try:
        for geo in GEOMETRIES:
            api.ipa_launch_config_set(m, n, geo)
            api.ipa_launch_config_set(m, n, geo, grad=False)
            got = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
            nll = api.ipa_nll(m, ev, theta).cpu().numpy()
            if ref is None:
                ref = (got, nll)
                f_ref, g_ref = O.nll_grad(O.Model("4d", 0.0, 15.0), cols, TH4)
                logl, _ = O.nll_grad_terms(O.Model("4d", 0.0, 15.0), cols, TH4)
                labs = math.fsum(np.abs(logl))
                G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, O.Model("4d", 0.0, 15.0), cols, TH4),
                                        labs)
            assert np.array_equal(got, ref[0]), geo
            assert np.array_equal(nll, ref[1]), geo
    finally:
        _restore_default(api, m, n)
        _restore_default(api, m, n, grad=False)


def test_segmented_geometries_and_solo_equal(env):
    """Many segments (ragged, one empty): every geometry gives the same bits,
    equal to each segment evaluated alone."""
    O, G, torch, api = env
    m = api.model_4d()
    sizes = [700, 0, 1, 20000, 513, 16384, 3000]
    n = sum(sizes)
    cols = synth.events_4d(n, 77)
    ev = G.to_dev(cols)
    off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    theta = torch.tensor(np.tile(TH4, (len(sizes), 1)) * (1 + 0.01 * np.arange(len(sizes)))[:, None],
                         device="cuda")
    ref = None
    try:
        for geo in GEOMETRIES:
            api.ipa_launch_config_set(m, n, geo, n_seg=len(sizes))
            got = api.ipa_nll_grad_segmented(m, ev, off, theta).cpu().numpy()
            if ref is None:
                ref = got
            assert np.array_equal(got, ref), geo
    finally:
        _restore_default(api, m, n, n_seg=len(sizes))
    for i, (a, b) in enumerate(zip(off[:-1].tolist(), off[1:].tolist())):
        sub = {k: v[a:b].clone() for k, v in ev.items()}
        solo = api.ipa_nll_grad(m, sub, theta[i].contiguous()).cpu().numpy()
        assert np.array_equal(solo, ref[i]), i


def test_autotune_picks_a_valid_geometry_and_keeps_results(env):
    O, G, torch, api = env
    m = api.model_4d()
    n = 300_000
    ev = G.to_dev(synth.events_4d(n, 5))
    theta = torch.tensor(TH4, device="cuda")
    before = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
    try:
        picked = api.ipa_autotune(m, ev, theta, grad=True)
        assert picked["warps_per_block"] in (1, 2, 4, 8)
        assert picked["warps_per_sm"] in (0, 64)
        assert picked["tiles_per_take"] in (1, 2, 4)
        assert 0.0 < picked["ms"] < 100.0
        now = api.ipa_launch_config_get(m, n)
        assert {k: now[k] for k in ("warps_per_block", "warps_per_sm", "tiles_per_take")} == \
            {k: picked[k] for k in ("warps_per_block", "warps_per_sm", "tiles_per_take")}
        after = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
        assert np.array_equal(before, after)
    finally:
        _restore_default(api, m, n)


def test_autotune_refuses_a_capturing_stream(env):
    O, G, torch, api = env
    m = api.model_4d()
    ev = G.to_dev(synth.events_4d(1000, 6))
    theta = torch.tensor(TH4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            try:
                api.ipa_autotune(m, ev, theta, stream=s)
            except api.IpaError as e:
                err = e
    assert err is not None and "IPA_ERR_BUSY" in str(err)


def test_batched_fit_is_unchanged_by_tuning(env):
    """The fitter's cached graph is re-captured after the geometry changes, and
    the fitted parameters do not move by a bit."""
    O, G, torch, api = env
    m = api.model_4d()
    n_fits, size = 16, 4000
    cols = synth.events_4d(n_fits * size, 9)
    ev = G.to_dev(cols)
    off = torch.arange(0, (n_fits + 1) * size, size, dtype=torch.int64, device="cuda")
    lo = [0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2]
    hi = [1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2]
    step = [0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2]
    params = [api.Param(float(TH4[i]), lo[i], hi[i], step[i]) for i in range(10)]
    start = torch.tensor(np.tile(TH4, (n_fits, 1)), device="cuda")
    r0 = api.ipa_fit_batch(m, ev, off, params, start.clone())
    try:
        api.ipa_launch_config_set(m, n_fits * size, {"warps_per_block": 8, "warps_per_sm": 64,
                                                     "tiles_per_take": 4}, n_seg=n_fits)
        r1 = api.ipa_fit_batch(m, ev, off, params, start.clone())
    finally:
        _restore_default(api, m, n_fits * size, n_seg=n_fits)
    for k in ("theta", "err", "nll", "status", "iters", "passes"):
        assert np.array_equal(r0[k].cpu().numpy(), r1[k].cpu().numpy()), k
