"""GPU parity of ipa_nll / ipa_nll_grad / ipa_nll_grad_segmented against the oracle.

Tolerances: NLL to 1e-12 relative (to sum |w log P|);
gradient to 1e-9 relative to max(|g_j|, condition scale of g_j) -- see
gpu_common.grad_scale -- and, against central finite differences of the GPU
NLL itself, to 1e-6.
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH1 = np.array([0.66, 0.045, 0.0, 0.1])
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def _parity(env, kind, n, seed, weighted, th, t_lo=None):
    O, G, torch, api = env
    if kind == "1d":
        t_lo = 0.3 if t_lo is None else t_lo
        m_o, m_g = O.Model("1d", t_lo, 15.0), api.model_1d(t_lo, 15.0)
        cols = {"t": synth.events_1d(n, seed, t_lo=t_lo)}
        if weighted:
            cols["w"] = synth.weights(n, seed + 1)
    else:
        t_lo = 0.0 if t_lo is None else t_lo
        m_o, m_g = O.Model("4d", t_lo, 15.0), api.model_4d(t_lo, 15.0)
        cols = synth.events_4d(n, seed, t_lo=t_lo, weighted=weighted)
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    got = api.ipa_nll_grad(m_g, ev, theta).cpu().numpy()
    nll_only = float(api.ipa_nll(m_g, ev, theta).cpu()[0])
    f_ref, g_ref = O.nll_grad(m_o, cols, th)
    logl, _ = O.nll_grad_terms(m_o, cols, th)
    labs = math.fsum(np.abs(logl)) if n else 1.0
    scale = G.grad_scale(O, m_o, cols, th) if n else np.zeros(th.size)
    G.assert_nll_grad_close(got, f_ref, g_ref, scale, labs)
    assert abs(nll_only - f_ref) <= 1e-12 * labs
    if n >= 100_000:
        G.report_margin(f"{kind} {n}", got, f_ref, g_ref, scale)
    return got


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 511, 512, 513, 1025, 4097, 100000])
@pytest.mark.parametrize("kind", ["1d", "4d"])
def test_parity_sizes(env, kind, n):
    _parity(env, kind, n, seed=n + 3, weighted=False, th=TH1 if kind == "1d" else TH4)


@pytest.mark.parametrize("kind", ["1d", "4d"])
def test_parity_weighted_and_off_truth(env, kind):
    th = (TH1 if kind == "1d" else TH4).copy()
    th[0], th[1], th[2] = 0.8, 0.06, 0.01
    if kind == "4d":
        th[4:10] = [0.45, 0.3, 2.5, -0.4, 0.15, 1.1]
    _parity(env, kind, 20000, seed=5, weighted=True, th=th, t_lo=0.0)


@pytest.mark.parametrize("kind", ["1d", "4d"])
@pytest.mark.parametrize("weighted", [False, True])
def test_parity_range_far_before_the_peak(env, kind, weighted):
    """A range starting 3 ps (67 sigma) before mu: the early events' Gaussian
    exponent -tau^2/(2 sigma^2) reaches -2200, below the integer exp's range,
    where the kernels clamp it at -705 (the Gaussian is then nothing against
    the exponential term); whole tiles, a ragged tail, against the oracle."""
    _parity(env, kind, 20_001, seed=41, weighted=weighted and kind == "4d", th=TH4 if kind == "4d" else TH1,
            t_lo=-3.0)


def test_parity_config2_full_size(env):
    """4D, 1e6 events (the headline workload), unweighted."""
    _parity(env, "4d", 1_000_000, seed=0, weighted=False, th=TH4)


def test_parity_config1_full_size(env):
    """1D, 1e5 events on [0.3, 15] ps."""
    _parity(env, "1d", 100_000, seed=0, weighted=False, th=TH1)


def test_gradient_vs_gpu_finite_differences(env):
    O, G, torch, api = env
    cols = synth.events_4d(50000, 11, weighted=True)
    ev = G.to_dev(cols)
    m = api.model_4d()
    th = TH4.copy()
    th[2] = 0.003
    g = api.ipa_nll_grad(m, ev, torch.tensor(th, device="cuda")).cpu().numpy()[1:]
    f0 = float(api.ipa_nll(m, ev, torch.tensor(th, device="cuda")).cpu()[0])
    for j in range(th.size):
        h = 1e-5 * max(abs(th[j]), 0.05)
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fp = float(api.ipa_nll(m, ev, torch.tensor(tp, device="cuda")).cpu()[0])
        fm = float(api.ipa_nll(m, ev, torch.tensor(tm, device="cuda")).cpu()[0])
        fd = (fp - fm) / (2 * h)
        noise = abs(f0) * 4e-16 / h
        assert abs(g[j] - fd) <= 1e-6 * max(abs(g[j]), abs(fd)) + noise + 1e-6, (j, g[j], fd)


def test_deterministic_and_segment_equals_solo(env):
    """Bitwise: repeated calls agree; each segment of a packed call equals the solo call."""
    O, G, torch, api = env
    m = api.model_4d()
    sizes = [0, 1, 700, 513, 20000, 3, 4096, 0, 12345]
    cols = synth.events_4d(sum(sizes), 21, weighted=True)
    ev = G.to_dev(cols)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(2)
    thetas = np.tile(TH4, (len(sizes), 1))
    thetas[:, 0] += rng.normal(0, 0.02, len(sizes))
    seg = api.ipa_nll_grad_segmented(m, ev, torch.tensor(off, device="cuda"),
                                     torch.tensor(thetas, device="cuda")).cpu().numpy()
    seg2 = api.ipa_nll_grad_segmented(m, ev, torch.tensor(off, device="cuda"),
                                      torch.tensor(thetas, device="cuda")).cpu().numpy()
    assert np.array_equal(seg, seg2)
    for s, (a, b) in enumerate(zip(off[:-1], off[1:])):
        sub = {k: v[a:b].clone() for k, v in ev.items()}   # fresh, 16-byte aligned
        solo = api.ipa_nll_grad(m, sub, torch.tensor(thetas[s], device="cuda")).cpu().numpy()
        assert np.array_equal(solo, seg[s]), s
        if b == a:
            assert np.all(seg[s] == 0.0)


def test_many_segments_equal_solo(env):
    """80 segments (the constants are then computed one thread per fit) against
    solo calls (one six-warp block per fit): bitwise equal, with every
    parameter moved so that every row of the constants is exercised."""
    O, G, torch, api = env
    m = api.model_4d()
    rng = np.random.default_rng(8)
    sizes = rng.integers(0, 3000, 80)
    cols = synth.events_4d(int(sizes.sum()), 22, weighted=True)
    ev = G.to_dev(cols)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    thetas = np.tile(TH4, (80, 1))
    thetas[:, 0] += rng.normal(0, 0.02, 80)
    thetas[:, 4] += rng.normal(0, 0.02, 80)
    thetas[:, 1] += rng.normal(0, 0.003, 80)
    thetas[:, 2] += rng.normal(0, 0.005, 80)
    thetas[:, 3] += rng.normal(0, 0.01, 80)
    thetas[:, 5] += rng.normal(0, 0.02, 80)
    thetas[:, 6:8] += rng.normal(0, 0.3, (80, 2))
    thetas[:, 8] += rng.normal(0, 0.01, 80)
    thetas[:, 9] += rng.normal(0, 0.3, 80)
    seg = api.ipa_nll_grad_segmented(m, ev, torch.tensor(off, device="cuda"),
                                     torch.tensor(thetas, device="cuda")).cpu().numpy()
    for s in (0, 1, 17, 41, 63, 79):
        a, b = off[s], off[s + 1]
        sub = {k: v[a:b].clone() for k, v in ev.items()}
        solo = api.ipa_nll_grad(m, sub, torch.tensor(thetas[s], device="cuda")).cpu().numpy()
        assert np.array_equal(solo, seg[s]), s


def test_misaligned_column_rejected(env):
    O, G, torch, api = env
    t = torch.zeros(101, dtype=torch.float64, device="cuda")
    with pytest.raises(api.IpaError, match="aligned"):
        api.ipa_nll(api.model_1d(), {"t": t[1:]}, torch.tensor(TH1, device="cuda"))


def test_large_weighted_sampled(env):
    """5e7 weighted 4D events (the large single-fit workload, ~2 GB): the full NLL+grad
    equals the sum over 50 segments of 1e6 (a property at any size), and three of
    those segments match the oracle."""
    O, G, torch, api = env
    n, k = 50_000_000, 50
    ev = G.to_dev(synth.events_4d(n, 5, weighted=True))
    m = api.model_4d()
    th = torch.tensor(TH4, device="cuda")
    full = api.ipa_nll_grad(m, ev, th).cpu().numpy()
    off = torch.arange(0, n + 1, n // k, dtype=torch.int64, device="cuda")
    seg = api.ipa_nll_grad_segmented(m, ev, off, th.repeat(k, 1)).cpu().numpy()
    tot = seg.sum(axis=0)
    assert abs(full[0] - tot[0]) <= 1e-12 * abs(full[0])
    np.testing.assert_allclose(full[1:], tot[1:], rtol=1e-9, atol=1e-9 * np.abs(seg[:, 1:]).sum(axis=0).max())
    mo = O.Model("4d", 0.0, 15.0)
    for s in (0, 17, 49):
        a, b = s * (n // k), (s + 1) * (n // k)
        cols = {key: v[a:b].cpu().numpy() for key, v in ev.items()}
        f_ref, g_ref = O.nll_grad(mo, cols, TH4)
        logl, _ = O.nll_grad_terms(mo, cols, TH4)
        G.assert_nll_grad_close(seg[s], f_ref, g_ref, G.grad_scale(O, mo, cols, TH4),
                                math.fsum(np.abs(logl)))
    del ev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind", ["1d", "4d"])
def test_weight_column_of_ones_equals_no_column(env, kind):
    """Events of weight exactly 1 take the unweighted path's log product, so a
    weight column of ones gives the NLL and gradient of no column bit for bit
    (the server stores ones for unweighted requests); other weights keep
    w log P and still match the oracle."""
    O, G, torch, api = env
    n = 30001
    if kind == "1d":
        m, th, cols = api.model_1d(0.3, 15.0), TH1, {"t": synth.events_1d(n, 8)}
    else:
        m, th, cols = api.model_4d(0.0, 15.0), TH4, synth.events_4d(n, 8)
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    plain = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
    ones = api.ipa_nll_grad(m, dict(ev, w=torch.ones(n, dtype=torch.float64, device="cuda")), theta).cpu().numpy()
    assert np.array_equal(plain, ones)
    # mixed: a third of the weights exactly 1, the rest Normal(1, 0.2)
    w = synth.weights(n, 9)
    w[::3] = 1.0
    got = api.ipa_nll_grad(m, dict(ev, w=torch.tensor(w, device="cuda")), theta).cpu().numpy()
    wc = dict(cols, w=w)
    m_o = O.Model(kind, 0.3 if kind == "1d" else 0.0, 15.0)
    f_ref, g_ref = O.nll_grad(m_o, wc, th)
    logl, _ = O.nll_grad_terms(m_o, wc, th)
    G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, m_o, wc, th), math.fsum(np.abs(logl)))


def _chunks(n):
    """The host entry point's chunking: k = clamp(floor(n / 2^20), 1, 16) pieces of
    ceil(ceil(n / k) / 512) * 512 events."""
    k = min(max(n // (1 << 20), 1), 16)
    per = -(-n // k)
    chunk = -(-per // 512) * 512
    return [(o, min(chunk, n - o)) for o in range(0, n, chunk)]


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("kind,n,weighted", [("4d", 1_000_000, False), ("4d", 300_001, True), ("1d", 1000, False),
                                             ("4d", 3_000_000, True), ("4d", 0, False)])
def test_host_entry_point(env, kind, n, weighted, pinned):
    """ipa_nll_grad_host: page-locked columns are read in place, so the result is
    bitwise ipa_nll_grad of the same events; pageable columns are staged in
    chunks and the result is the sum, in chunk order, of ipa_nll_grad over each
    chunk (bitwise).  Both match the oracle (up to 4e5 events)."""
    O, G, torch, api = env
    if kind == "1d":
        m_o, m_g = O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0)
        cols = {"t": synth.events_1d(n, 5)}
        th = TH1
    else:
        m_o, m_g = O.Model("4d", 0.0, 15.0), api.model_4d(0.0, 15.0)
        cols = synth.events_4d(n, 6, weighted=weighted)
        th = TH4 * 1.01
    host = {k: (torch.tensor(v).pin_memory() if pinned else torch.tensor(v)) for k, v in cols.items()}
    theta = torch.tensor(th, device="cuda")
    got = api.ipa_nll_grad_host(m_g, host, theta).cpu().numpy()
    again = api.ipa_nll_grad_host(m_g, host, theta).cpu().numpy()
    assert np.array_equal(got, again)
    if n == 0:
        assert np.all(got == 0.0)
        return
    if pinned:
        ref = api.ipa_nll_grad(m_g, G.to_dev(cols), theta).cpu().numpy()
    else:
        ref = np.zeros(th.size + 1)
        for o, ln in _chunks(n):
            part = api.ipa_nll_grad(m_g, G.to_dev({k: v[o:o + ln] for k, v in cols.items()}), theta).cpu().numpy()
            ref = ref + part
    assert np.array_equal(got, ref)
    if n <= 400_000:
        f_ref, g_ref = O.nll_grad(m_o, cols, th)
        logl, _ = O.nll_grad_terms(m_o, cols, th)
        G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, m_o, cols, th), math.fsum(np.abs(logl)))


def test_host_entry_point_rejects_device_and_mixed_columns(env):
    O, G, torch, api = env
    m = api.model_1d(0.3, 15.0)
    theta = torch.tensor(TH1, device="cuda")
    with pytest.raises(api.IpaError):
        api.ipa_nll_grad_host(m, {"t": torch.zeros(10, dtype=torch.float64, device="cuda")}, theta)
    with pytest.raises(api.IpaError):
        api.ipa_nll_grad_host(m, {"t": torch.zeros(10, dtype=torch.float64), "w": torch.zeros(9, dtype=torch.float64)},
                              theta)
