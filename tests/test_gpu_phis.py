"""GPU parity of the time-dependent angular model with tagging
(IPA_MODEL_PHIS) against the oracle (oracle/phis.py).

* NLL to 1e-12 relative (to sum |w log P|) and gradient to 1e-9 relative to
  max(|g_j|, the condition scale of g_j) over sizes spanning several tiles and
  a ragged tail, parameter points (phi_s = 0, omega = 1/2, a large S wave, a
  range before the resolution peak), weighted and not, the raw and the cached
  angular basis;
* a category of one flavour (normalisation over the selected tag alone);
* the gradient against fourth-order central differences of the GPU NLL;
* segments bitwise equal to solo calls;
* a batched fit within 1e-6 sigma of the oracle's fit on events drawn from the
  model (accept-reject with numpy's generator in the test).
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.8, 0.3, 0.8, 0.0])
THETAS = {
    "truth": TH,
    "phi_zero": np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.0, 0.3, 1.0, 0.0]),
    "half_mistag": np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.8, 0.5, 0.8,
                             0.0]),
    "large_s_wave": np.array([0.7, 0.06, 0.01, 0.2, 0.4, 0.3, 2.0, -1.0, 0.3, -1.2, -0.1, 12.0, -2.0, 0.1, 0.5, 0.0]),
    "no_s_p_overlap": np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.1, 0.3, 0.085, 17.77, 0.8, 0.3, 0.0,
                                0.0]),
}


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from oracle import phis
    from paper_1706_01420_gb300 import api
    return oracle, phis, G, torch, api


def grad_scale(F, m, ev, th):
    """Condition scale: sum over events of |w| / P times the sum of the absolute
    values of the per-event derivative pieces (here bounded by the absolute
    derivative rows of the rate, plus |rate dlnN| and, for f_b, |rate|/N + 1/V)."""
    th = np.asarray(th, dtype=np.float64)
    w = np.abs(np.asarray(ev["w"])) if ev.get("w") is not None else np.ones(len(ev["t"]))
    N, dN = F.norm_grad(m, th)
    R, dR = F.rate_grad(m, ev, th)
    P = F.pdf(m, ev, th)
    cs = (1 - th[3]) / N
    r = w / P
    out = np.zeros(16)
    for j in range(15):
        if j == 3:
            out[j] = math.fsum(r * (np.abs(R) / N + 1 / F.volume(m, th)))
        else:
            # each derivative row is a sum of ~10 angular terms of either sign:
            # allow the sum of their magnitudes through a factor 10 on |dR|
            out[j] = cs * math.fsum(r * (10.0 * np.abs(dR[j]) + np.abs(R) * abs(dN[j] / N)))
    return out


def _parity(env, n, seed, th, weighted=False, t_lo=0.0, cached=False, tag=0.0):
    O, F, G, torch, api = env
    m_o, m_g = O.Model("phis", t_lo, 15.0), api.model_phis(t_lo, 15.0)
    cols = synth.events_phis(n, seed, t_lo=t_lo, weighted=weighted)
    if tag:
        # a category of one flavour: every event carries the selected tag
        th = th.copy()
        th[15] = tag
        cols["q"] = np.full(n, tag)
    ev = G.to_dev(cols)
    if cached and n:
        ev["fk"] = api.ipa_angular_basis(m_g, ev)
    theta = torch.tensor(th, device="cuda")
    got = api.ipa_nll_grad(m_g, ev, theta).cpu().numpy()
    nll_only = float(api.ipa_nll(m_g, ev, theta).cpu()[0])
    f_ref, g_ref = F.nll_grad(m_o, cols, th)
    logl, _ = F.nll_grad_terms(m_o, cols, th)
    labs = math.fsum(np.abs(logl)) if n else 1.0
    scale = grad_scale(F, m_o, cols, th) if n else np.zeros(16)
    G.assert_nll_grad_close(got, f_ref, g_ref, scale, labs)
    assert abs(nll_only - f_ref) <= 1e-12 * labs
    return got


@pytest.mark.parametrize("n", [0, 1, 513, 4097, 20000])
def test_parity_sizes(env, n):
    _parity(env, n, seed=n + 5, th=TH)


@pytest.mark.parametrize("name", sorted(THETAS))
@pytest.mark.parametrize("weighted", [False, True])
def test_parity_parameters(env, name, weighted):
    _parity(env, 12000, seed=3, th=THETAS[name], weighted=weighted)


@pytest.mark.parametrize("tag", [1.0, -1.0])
@pytest.mark.parametrize("name", ["truth", "large_s_wave"])
def test_parity_one_tag_normalisation(env, name, tag):
    _parity(env, 12000, seed=9, th=THETAS[name], weighted=True, tag=tag)
    _parity(env, 4097, seed=10, th=THETAS[name], tag=tag, cached=True)


def test_parity_pole_angles_and_a_huge_weight(env):
    """Angles within 2^-17 of the poles (|cos| = 1 - 1e-7, 1 - 2^-18) and phi =
    +-pi, where the angular functions lose relative precision, and one event of
    weight 1e7 that dominates the weighted sums: against the oracle, weighted
    and not, with the tolerances of the other parity tests."""
    O, F, G, torch, api = env
    m_o, m_g = O.Model("phis", 0.0, 15.0), api.model_phis(0.0, 15.0)
    for weighted in (False, True):
        cols = synth.events_phis(4096, 31, weighted=weighted)
        cols["ck"][::97] = 1.0 - 1e-7
        cols["ck"][5::97] = -(1.0 - 1e-7)
        cols["cl"][11::89] = 1.0 - 2.0 ** -18
        cols["phi"][3::53] = np.pi
        cols["phi"][7::53] = -np.pi
        if weighted:
            cols["w"][1234] = 1.0e7
        ev = G.to_dev(cols)
        theta = torch.tensor(TH, device="cuda")
        got = api.ipa_nll_grad(m_g, ev, theta).cpu().numpy()
        f_ref, g_ref = F.nll_grad(m_o, cols, TH)
        logl, _ = F.nll_grad_terms(m_o, cols, TH)
        G.assert_nll_grad_close(got, f_ref, g_ref, grad_scale(F, m_o, cols, TH), math.fsum(np.abs(logl)))


def test_parity_cached_basis_and_early_range(env):
    _parity(env, 12000, seed=4, th=TH, cached=True)
    _parity(env, 12000, seed=6, th=THETAS["large_s_wave"], weighted=True, t_lo=-0.3, cached=True)


def test_gradient_matches_finite_differences(env):
    O, F, G, torch, api = env
    m = api.model_phis(0.0, 15.0)
    ev = G.to_dev(synth.events_phis(30000, 8, weighted=True))
    base = TH + np.array([0.01, 0.002, 0.001, 0.02, 0.01, -0.01, 0.05, -0.05, 0.01, 0.1, 0.01, 0.05, 0.05, 0.01,
                          -0.05, 0.0])
    for Q in (0.0, -1.0):
        th = base.copy()
        th[15] = Q
        e = ev if Q == 0.0 else dict(ev, q=torch.full_like(ev["q"], Q))
        g = api.ipa_nll_grad(m, e, torch.tensor(th, device="cuda")).cpu().numpy()[1:]
        assert g[15] == 0.0

        def f(j, d):
            tt = th.copy()
            tt[j] += d
            return float(api.ipa_nll(m, e, torch.tensor(tt, device="cuda")).cpu()[0])

        for j in range(15):
            # steps of 1e-5 of the parameter's scale (at least 0.1): roundoff of the
            # 3e4-event NLL stays below the 1e-6 bound
            h = 1e-5 * max(abs(th[j]), 0.1)
            fd = (8.0 * (f(j, h) - f(j, -h)) - (f(j, 2 * h) - f(j, -2 * h))) / (12.0 * h)
            assert abs(fd - g[j]) <= 1e-6 * max(abs(g[j]), 1.0), (Q, j, fd, g[j])


def test_segments_equal_solo(env):
    O, F, G, torch, api = env
    m = api.model_phis(0.0, 15.0)
    sizes = [900, 0, 4000, 1, 2049]
    parts = [synth.events_phis(k, 20 + i, weighted=True) for i, k in enumerate(sizes)]
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
    """72 segments (the record then computed one thread per segment) against
    solo calls (one block per segment): bitwise equal, every parameter moved and
    the normalisation over both tags, the tag +1 and the tag -1 in turn (the
    complex edges of the one-tag record in both layouts)."""
    O, F, G, torch, api = env
    m = api.model_phis(0.0, 15.0)
    rng = np.random.default_rng(32)
    n_seg = 72
    sizes = rng.integers(0, 1200, n_seg)
    parts = [synth.events_phis(int(k), 200 + i, weighted=True) for i, k in enumerate(sizes)]
    cols = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    ev = G.to_dev(cols)
    names = sorted(THETAS)
    ths = np.stack([THETAS[names[i % len(names)]] for i in range(n_seg)])
    ths[:, 0] += rng.normal(0, 0.02, n_seg)
    ths[:, 1] += rng.normal(0, 0.003, n_seg)
    ths[:, 2] += rng.normal(0, 0.005, n_seg)
    ths[:, 4:6] += rng.normal(0, 0.01, (n_seg, 2))
    ths[:, 6:8] += rng.normal(0, 0.3, (n_seg, 2))
    ths[:, 8] = np.clip(ths[:, 8] + rng.normal(0, 0.01, n_seg), 0.0, 1.0)
    ths[:, 9] += rng.normal(0, 0.3, n_seg)
    ths[:, 10] += rng.normal(0, 0.01, n_seg)
    ths[:, 11] += rng.normal(0, 0.2, n_seg)
    ths[:, 12] += rng.normal(0, 0.3, n_seg)
    ths[:, 13] = np.clip(ths[:, 13] + rng.normal(0, 0.02, n_seg), 0.0, 0.5)
    ths[:, 15] = np.array([0.0, 1.0, -1.0])[np.arange(n_seg) % 3]
    off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    seg = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(ths, device="cuda")).cpu().numpy()
    for i in (0, 1, 2, 31, 64, 70, 71):
        solo = api.ipa_nll_grad(m, G.to_dev(parts[i]), torch.tensor(ths[i], device="cuda")).cpu().numpy()
        assert np.array_equal(seg[i], solo), i


def _sample(F, m, th, n, seed):
    """Events of the model by accept-reject (uniform t, angles, tag; the bound is
    1.5 x the largest density of 2e5 candidates, checked against every candidate)."""
    rng = np.random.default_rng(seed)

    def cand(k):
        return {"t": rng.uniform(m.t_lo, m.t_hi, k), "ck": rng.uniform(-1, 1, k), "cl": rng.uniform(-1, 1, k),
                "phi": rng.uniform(-math.pi, math.pi, k), "q": np.where(rng.uniform(size=k) < 0.5, 1.0, -1.0)}

    bound = 1.5 * F.pdf(m, cand(200000), th).max()
    out = {k: [] for k in ("t", "ck", "cl", "phi", "q")}
    got = 0
    while got < n:
        c = cand(200000)
        p = F.pdf(m, c, th)
        assert p.max() < bound
        keep = rng.uniform(0, bound, p.size) < p
        for k in out:
            out[k].append(c[k][keep])
        got += int(keep.sum())
    return {k: np.concatenate(v)[:n] for k, v in out.items()}


def test_fit_matches_oracle_and_batch_equals_solo(env):
    """sigma, mu, omega, C_SP and the tag selector held; the eleven others free."""
    O, F, G, torch, api = env
    m_o, m = O.Model("phis", 0.0, 15.0), api.model_phis(0.0, 15.0)
    toys = [_sample(F, m_o, TH, 6000, 100 + k) for k in range(3)]
    free = [0, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12]
    lo = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2, -0.5, 10.0, -3.1, 0.0, 0.0, -1.0])
    hi = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2, 0.5, 25.0, 3.1, 0.5, 1.0, 1.0])
    step = (hi - lo) / 50
    start = TH.copy()
    params = [api.Param(float(start[i]), float(lo[i]), float(hi[i]), float(step[i]), fixed=i not in free)
              for i in range(16)]
    sizes = [t["t"].size for t in toys]

    def fit(sel):
        c = {k: np.concatenate([toys[i][k] for i in sel]) for k in toys[0]}
        off = torch.tensor(np.concatenate([[0], np.cumsum([sizes[i] for i in sel])]), dtype=torch.int64,
                           device="cuda")
        theta = torch.tensor(np.tile(start, (len(sel), 1)), device="cuda")
        r = api.ipa_fit_batch(m, G.to_dev(c), off, params, theta, max_iter=300, tol=1e-9)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in r.items()}

    batch = fit([0, 1, 2])
    solo = fit([2])
    for key in ("theta", "err", "nll", "status", "iters"):
        assert np.array_equal(solo[key][0], batch[key][2]), key
    ref = O.fit(m_o, toys[0], start, free, lo=lo, hi=hi, tol=1e-10, max_iter=100)
    assert batch["status"][0] in (0, 2) and ref.status == "CONVERGED"
    for j in free:
        assert abs(batch["theta"][0, j] - ref.theta[j]) < 1e-6 * ref.err[j], (j, batch["theta"][0, j], ref.theta[j])
        assert batch["err"][0, j] == pytest.approx(ref.err[j], rel=1e-3)
    assert batch["nll"][0] == pytest.approx(ref.nll, rel=1e-12)


@pytest.mark.parametrize("Q", [0.0, 1.0, -1.0])
def test_toys_bit_exact(env, Q):
    """The generator's streams equal the oracle's toy_one bit for bit (both tags
    drawn, or one selected), including an empty toy and one without background."""
    O, F, G, torch, api = env
    m_o, m_g = O.Model("phis", 0.0, 15.0), api.model_phis(0.0, 15.0)
    th = TH.copy()
    th[15] = Q
    n_sig = np.array([2000, 0, 700], dtype=np.int64)
    n_bkg = np.array([200, 30, 0], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(n_sig + n_bkg)[:-1]])
    cap = int((n_sig + n_bkg).sum())
    out = {k: torch.empty(cap, dtype=torch.float64, device="cuda") for k in ("t", "ck", "cl", "phi", "q")}
    dv = lambda a: torch.tensor(a, dtype=torch.int64, device="cuda")
    api.ipa_toygen(m_g, torch.tensor(th, device="cuda"), 2024, dv(n_sig), dv(n_bkg), dv(off), out)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for k in range(3):
        ref = F.toy_one(m_o, th, 2024, k, int(n_sig[k]), int(n_bkg[k]))
        sl = slice(int(off[k]), int(off[k] + n_sig[k] + n_bkg[k]))
        for col in ("t", "ck", "cl", "phi", "q"):
            assert np.array_equal(got[col][sl], ref[col]), (k, col)


def test_parity_full_size_bench_workload(env):
    """The phi_s workload of the benchmark at its full size: 1e6 synthetic
    events (seed 11) at the benchmark's parameters, NLL and gradient against the
    oracle, raw and with the cached angular basis."""
    O, F, G, torch, api = env
    th = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.8, 0.3, 0.8, 0.0])
    m_o, m_g = O.Model("phis", 0.0, 15.0), api.model_phis(0.0, 15.0)
    cols = synth.events_phis(1_000_000, 11)
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    got = api.ipa_nll_grad(m_g, ev, theta).cpu().numpy()
    cached = api.ipa_nll_grad(m_g, dict(ev, fk=api.ipa_angular_basis(m_g, ev)), theta).cpu().numpy()
    f_ref, g_ref = F.nll_grad(m_o, cols, th)
    logl, _ = F.nll_grad_terms(m_o, cols, th)
    scale = grad_scale(F, m_o, cols, th)
    for out in (got, cached):
        G.assert_nll_grad_close(out, f_ref, g_ref, scale, math.fsum(np.abs(logl)))
    G.report_margin("phis 1e6", got, f_ref, g_ref, scale)
