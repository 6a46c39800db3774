"""GPU parity of the flavour-tagged model (IPA_MODEL_TAGGED1D) against the
oracle (oracle/tagged.py).

* ipa_faddeeva against scipy.special.wofz (the oracle's Faddeeva function),
  and the exact symmetry w(-conj z) = conj w(z);
* NLL to 1e-12 relative (to sum |w log P|) and gradient to 1e-9 relative to
  max(|g_j|, condition scale of g_j) over sizes that span several tiles and a
  ragged tail, several parameter points (phi_s = 0, DG < 0, a wide resolution
  with fast oscillation, a range that starts before the resolution peak),
  weighted and unweighted; the gradient against central differences of the
  GPU NLL to 1e-6; segments bitwise equal to solo calls;
* toys bit-exact against the oracle's generator; a batched fit within 1e-6
  sigma of the oracle's fit.
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TRUTH = np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.8, 0.3])
THETAS = {
    "truth": TRUTH,
    "dg_negative": np.array([1.2, 0.08, 0.02, 0.3, -0.1, 5.0, -2.0, 0.1]),
    "fast_mixing": np.array([0.5, 0.03, -0.01, 0.0, 0.2, 25.0, 1.57, 0.45]),
    "phi_zero": np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.0, 0.3]),
    "wide_resolution": np.array([0.7, 0.2, 0.05, 0.2, 0.1, 30.0, 2.5, 0.05]),
}


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from oracle import tagged
    from paper_1706_01420_gb300 import api
    return oracle, tagged, G, torch, api


def _parity(env, n, seed, th, weighted=False, t_lo=0.0):
    O, T, G, torch, api = env
    m_o, m_g = O.Model("tag", t_lo, 15.0), api.model_tagged(t_lo, 15.0)
    cols = synth.events_tagged(n, seed, t_lo=t_lo, weighted=weighted)
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    got = api.ipa_nll_grad(m_g, ev, theta).cpu().numpy()
    nll_only = float(api.ipa_nll(m_g, ev, theta).cpu()[0])
    f_ref, g_ref = T.nll_grad(m_o, cols, th)
    logl, _ = T.nll_grad_terms(m_o, cols, th)
    labs = math.fsum(np.abs(logl)) if n else 1.0
    scale = G.grad_scale_tagged(O, T, m_o, cols, th) if n else np.zeros(8)
    G.assert_nll_grad_close(got, f_ref, g_ref, scale, labs)
    assert abs(nll_only - f_ref) <= 1e-12 * labs
    return got


def test_faddeeva_matches_scipy(env):
    from scipy.special import wofz
    O, T, G, torch, api = env
    x = np.concatenate([np.linspace(-8, 8, 81), [0.565, -0.565, 4.24, 1e-3, -1e-3]])
    y = np.concatenate([np.linspace(0, 20, 81), [1e-3, 6.3, 50.0, 300.0, 1e4]])
    X, Y = np.meshgrid(x, y)
    z = (X + 1j * Y).ravel()
    # lower half plane near the axis (the reflection formula)
    xl, yl = np.meshgrid(np.linspace(-2.5, 2.5, 21), np.linspace(-2.5, -0.05, 11))
    z = np.concatenate([z, (xl + 1j * yl).ravel()])
    w = api.ipa_faddeeva(torch.tensor(z, device="cuda")).cpu().numpy()
    ref = wofz(z)
    rel = np.abs(w - ref) / np.abs(ref)
    # scipy's own error reaches ~2e-14 near the real axis at large |Re z|
    assert rel.max() < 4e-14, (rel.max(), z[np.argmax(rel)])
    # in the region the model uses (|Re z| <= 4.5, Im z >= 0) both are within a few 1e-15
    near = (np.abs(z.real) <= 4.5) & (z.imag >= 0)
    assert rel[near].max() < 1e-14
    # w(-conj z) = conj w(z) holds exactly in the upper half plane
    up = z[z.imag >= 0]
    a = api.ipa_faddeeva(torch.tensor(up, device="cuda")).cpu().numpy()
    b = api.ipa_faddeeva(torch.tensor(-np.conj(up), device="cuda")).cpu().numpy()
    assert np.array_equal(a, np.conj(b))


def test_faddeeva_on_imaginary_axis_is_erfcx(env):
    """w(i y) = erfcx(y) for real y >= 0 (the real-rate case of the convolution)."""
    from scipy.special import erfcx
    O, T, G, torch, api = env
    y = np.concatenate([np.linspace(0, 6, 61), [10.0, 40.0, 1e3]])
    w = api.ipa_faddeeva(torch.tensor(1j * y, device="cuda")).cpu().numpy()
    assert np.all(np.abs(w.imag) <= 1e-16 * np.abs(w.real))
    np.testing.assert_allclose(w.real, erfcx(y), rtol=2e-15)


@pytest.mark.parametrize("n", [0, 1, 33, 512, 513, 4097, 30000])
def test_parity_sizes(env, n):
    _parity(env, n, seed=n + 11, th=TRUTH)


@pytest.mark.parametrize("name", sorted(THETAS))
@pytest.mark.parametrize("weighted", [False, True])
def test_parity_parameters(env, name, weighted):
    _parity(env, 20000, seed=7, th=THETAS[name], weighted=weighted)


def test_parity_range_before_the_peak(env):
    """t_lo - mu = -0.3 ps: events left of the resolution peak (Re u > 0 branch)."""
    _parity(env, 20000, seed=8, th=THETAS["wide_resolution"], t_lo=-0.3)
    _parity(env, 20000, seed=9, th=TRUTH, t_lo=-0.3, weighted=True)


def test_parity_range_far_before_the_peak(env):
    """t_lo - mu = -3 ps (67 sigma): the Gaussian exponent of the earliest events
    is below the integer exp's range and clamped at -705 (the Gaussian is then
    nothing against the exponential terms)."""
    _parity(env, 20001, seed=12, th=TRUTH, t_lo=-3.0)
    _parity(env, 20001, seed=13, th=TRUTH, t_lo=-3.0, weighted=True)


def test_gradient_matches_finite_differences(env):
    O, T, G, torch, api = env
    m = api.model_tagged(0.0, 15.0)
    ev = G.to_dev(synth.events_tagged(50000, 3, weighted=True))
    th = TRUTH + np.array([0.01, 0.002, 0.001, 0.02, 0.01, 0.05, 0.05, 0.01])
    g = api.ipa_nll_grad(m, ev, torch.tensor(th, device="cuda")).cpu().numpy()[1:]

    def f(j, d):
        tt = th.copy()
        tt[j] += d
        return float(api.ipa_nll(m, ev, torch.tensor(tt, device="cuda")).cpu()[0])

    # fourth-order central differences: the NLL's third derivative in Dm grows
    # like t^3 (the phase Dm t), which puts the h^2 error of the three-point
    # rule at 1e-6 of the derivative for h = 1e-5 Dm
    for j in range(8):
        h = 1e-5 * max(abs(th[j]), 1e-2)
        fd = (8.0 * (f(j, h) - f(j, -h)) - (f(j, 2 * h) - f(j, -2 * h))) / (12.0 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(abs(g[j]), 1.0), (j, fd, g[j])


def test_segments_equal_solo(env):
    O, T, G, torch, api = env
    m = api.model_tagged(0.0, 15.0)
    sizes = [700, 0, 5000, 1, 2049]
    parts = [synth.events_tagged(k, 20 + i, weighted=True) for i, k in enumerate(sizes)]
    cols = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    ev = G.to_dev(cols)
    names = sorted(THETAS)
    ths = np.stack([THETAS[names[i % len(names)]] for i in range(len(sizes))])
    off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    seg = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(ths, device="cuda")).cpu().numpy()
    for i, p in enumerate(parts):
        solo = api.ipa_nll_grad(m, G.to_dev(p), torch.tensor(ths[i], device="cuda")).cpu().numpy()
        assert np.array_equal(seg[i], solo), i


def test_many_segments_equal_solo(env):
    """80 segments (the record then computed one thread per segment) against
    solo calls (one block per segment): bitwise equal, every parameter moved so
    that every field of the record is exercised."""
    O, T, G, torch, api = env
    m = api.model_tagged(0.0, 15.0)
    rng = np.random.default_rng(31)
    n_seg = 80
    sizes = rng.integers(0, 1500, n_seg)
    parts = [synth.events_tagged(int(k), 100 + i, weighted=True) for i, k in enumerate(sizes)]
    cols = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    ev = G.to_dev(cols)
    names = sorted(THETAS)
    ths = np.stack([THETAS[names[i % len(names)]] for i in range(n_seg)])
    ths[:, 0] += rng.normal(0, 0.02, n_seg)
    ths[:, 1] += rng.normal(0, 0.003, n_seg)
    ths[:, 2] += rng.normal(0, 0.005, n_seg)
    ths[:, 3] = np.clip(ths[:, 3] + rng.normal(0, 0.01, n_seg), 0.0, 1.0)
    ths[:, 4] += rng.normal(0, 0.01, n_seg)
    ths[:, 5] += rng.normal(0, 0.2, n_seg)
    ths[:, 6] += rng.normal(0, 0.3, n_seg)
    ths[:, 7] = np.clip(ths[:, 7] + rng.normal(0, 0.02, n_seg), 0.0, 0.5)
    off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    seg = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(ths, device="cuda")).cpu().numpy()
    for i in (0, 1, 23, 47, 64, 79):
        solo = api.ipa_nll_grad(m, G.to_dev(parts[i]), torch.tensor(ths[i], device="cuda")).cpu().numpy()
        assert np.array_equal(seg[i], solo), i


@pytest.mark.parametrize("th", [TRUTH, THETAS["fast_mixing"]], ids=["truth", "fast_mixing"])
def test_toys_bit_exact(env, th):
    O, T, G, torch, api = env
    m_o, m_g = O.Model("tag", 0.0, 15.0), api.model_tagged(0.0, 15.0)
    n_sig = np.array([3000, 0, 1500], dtype=np.int64)
    n_bkg = np.array([300, 40, 0], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(n_sig + n_bkg)[:-1]])
    cap = int((n_sig + n_bkg).sum())
    out = {"t": torch.empty(cap, dtype=torch.float64, device="cuda"),
           "q": torch.empty(cap, dtype=torch.float64, device="cuda")}
    dv = lambda a: torch.tensor(a, dtype=torch.int64, device="cuda")
    api.ipa_toygen(m_g, torch.tensor(th, device="cuda"), 12345, dv(n_sig), dv(n_bkg), dv(off), out)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for k in range(3):
        ref = O.toy_one(m_o, th, 12345, k, int(n_sig[k]), int(n_bkg[k]))
        sl = slice(int(off[k]), int(off[k] + n_sig[k] + n_bkg[k]))
        assert np.array_equal(got["t"][sl], ref["t"]), k
        assert np.array_equal(got["q"][sl], ref["q"]), k


def test_fit_matches_oracle_and_batch_equals_solo(env):
    """omega is held (the tagged term measures (1 - 2 omega) sin phi_s); sigma and
    mu are held as in the 1D fits (the resolution leaves little trace)."""
    O, T, G, torch, api = env
    m_o, m = O.Model("tag", 0.0, 15.0), api.model_tagged(0.0, 15.0)
    toys = [O.toy_one(m_o, TRUTH, 4, k, 36000, 4000) for k in range(3)]
    free = [0, 3, 4, 5, 6]
    lo = np.array([0.3, 0.01, -0.1, 0.0, -0.5, 10.0, -3.1, 0.0])
    hi = np.array([1.5, 0.2, 0.1, 0.5, 0.5, 25.0, 3.1, 0.5])
    step = np.array([0.01, 0.003, 0.002, 0.005, 0.02, 0.05, 0.1, 0.01])
    start = TRUTH * 1.01
    params = [api.Param(float(start[i]), float(lo[i]), float(hi[i]), float(step[i]), fixed=i not in free)
              for i in range(8)]
    sizes = [t["t"].size for t in toys]
    cols = {k: np.concatenate([t[k] for t in toys]) for k in toys[0]}

    def fit(sel):
        c = {k: np.concatenate([toys[i][k] for i in sel]) for k in toys[0]}
        s = [sizes[i] for i in sel]
        off = torch.tensor(np.concatenate([[0], np.cumsum(s)]), dtype=torch.int64, device="cuda")
        theta = torch.tensor(np.tile(start, (len(sel), 1)), device="cuda")
        r = api.ipa_fit_batch(m, G.to_dev(c), off, params, theta, max_iter=200, tol=1e-9)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in r.items()}

    batch = fit([0, 1, 2])
    solo = fit([1])
    for key in ("theta", "err", "nll", "status", "iters"):
        assert np.array_equal(solo[key][0], batch[key][1]), key
    ref = O.fit(m_o, toys[0], start, free, lo=lo, hi=hi, tol=1e-10, max_iter=100)
    assert batch["status"][0] == 0 and ref.status == "CONVERGED"
    for j in free:
        assert abs(batch["theta"][0, j] - ref.theta[j]) < 1e-6 * ref.err[j], (j, batch["theta"][0, j], ref.theta[j])
        assert batch["err"][0, j] == pytest.approx(ref.err[j], rel=1e-3)
    assert batch["nll"][0] == pytest.approx(ref.nll, rel=1e-12)
    del cols


def test_parity_full_size_bench_workload(env):
    """The tagged workload of the benchmark at its full size: 50 toys of 2e4
    events (1.8e4 signal, 2e3 background, seed 7) drawn by the oracle's
    generator (bit for bit the events ipa_toygen writes), NLL and gradient
    against the oracle at the truth."""
    O, T, G, torch, api = env
    m_o, m_g = O.Model("tag", 0.0, 15.0), api.model_tagged(0.0, 15.0)
    toys = [T.toy_one(m_o, TRUTH, 7, k, 18000, 2000) for k in range(50)]
    cols = {k: np.concatenate([t[k] for t in toys]) for k in toys[0]}
    ev = G.to_dev(cols)
    got = api.ipa_nll_grad(m_g, ev, torch.tensor(TRUTH, device="cuda")).cpu().numpy()
    f_ref, g_ref = T.nll_grad(m_o, cols, TRUTH)
    logl, _ = T.nll_grad_terms(m_o, cols, TRUTH)
    scale = G.grad_scale_tagged(O, T, m_o, cols, TRUTH)
    G.assert_nll_grad_close(got, f_ref, g_ref, scale, math.fsum(np.abs(logl)))
    G.report_margin("tagged 1e6", got, f_ref, g_ref, scale)
