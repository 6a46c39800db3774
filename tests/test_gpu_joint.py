"""GPU parity of the simultaneous fit over categories (ipa_nll_grad_joint,
ipa_fit_joint) against the oracle (oracle/joint.py).

* the joint NLL and gradient to 1e-12 / 1e-9 (relative to the condition scale
  of each component, summed over the categories that feed it): the 4D model
  with shared, per-category and constant parameters, an empty category and
  ragged sizes; the phi_s model in twelve categories, six m(KK) bins times two
  flavours (per-bin F_S and delta_S, per-bin C_SP constants, each flavour
  normalised over its own tag: Sec. 4, Example 2);
* the joint result is bitwise the fixed-order sum (categories ascending, then
  model parameters) of ipa_nll_grad_segmented at the categories' parameters;
* joint fits within 1e-6 sigma of the oracle's joint fit (4D in four
  categories; the phi_s model in six one-flavour categories), errors within
  1e-3, and a batch of joint fits bitwise equal to each fit alone;
* HESSE of joint fits (ipa_hesse_joint): covariance in units of the errors
  within 2e-3 of the inverse of the oracle's Hessian, errors within 1e-3;
  MINOS of joint fits (ipa_minos_joint) within 1e-5 sigma of the oracle's
  profile-likelihood roots (a shared and a per-category parameter).
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

# C_SP of six m(KK) bins: synthetic values of the usual size (the overlap of
# the S- and P-wave lineshapes in a bin falls below 1 away from the phi peak)
CSP = (0.96, 0.93, 0.88, 0.90, 0.95, 0.97)


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from oracle import joint, phis
    from paper_1706_01420_gb300 import api
    return oracle, joint, phis, G, torch, api


def _pack(cats_per_fit):
    """Columns of all categories of all fits back to back, and the offsets."""
    flat = [c for cats in cats_per_fit for c in cats]
    cols = {k: np.concatenate([c[k] for c in flat]) for k in flat[0]}
    off = np.concatenate([[0], np.cumsum([c["t"].size for c in flat])]).astype(np.int64)
    return cols, off


def _scale(O, F, m, ev, th):
    """Per-parameter condition scale of one category's gradient."""
    from tests import gpu_common as G
    if m.kind == "phis":
        from tests.test_gpu_phis import grad_scale
        return grad_scale(F, m, ev, th)
    return G.grad_scale(O, m, ev, th)


def _check_parity(env, m_o, m_g, cats_per_fit, jmap, value, thetas):
    O, J, F, G, torch, api = env
    joint = api.Joint(jmap, value)
    cols, off = _pack(cats_per_fit)
    ev = G.to_dev(cols)
    offd = torch.tensor(off, device="cuda")
    got = api.ipa_nll_grad_joint(m_g, ev, offd, joint, torch.tensor(np.stack(thetas), device="cuda"))
    got = got.cpu().numpy()
    # fixed-order sum of the segmented results at the categories' parameters
    ths = np.concatenate([J.category_thetas(jmap, value, th) for th in thetas])
    seg = api.ipa_nll_grad_segmented(m_g, ev, offd, torch.tensor(ths, device="cuda")).cpu().numpy()
    n_cat = len(jmap)
    jm = np.asarray(jmap)
    for i, (cats, th) in enumerate(zip(cats_per_fit, thetas)):
        f = 0.0
        g = np.zeros(joint.n_joint)
        for c in range(n_cat):
            r = seg[i * n_cat + c]
            f += r[0]
            for p in range(jm.shape[1]):
                if jm[c, p] >= 0:
                    g[jm[c, p]] += r[1 + p]
        assert got[i, 0] == f
        assert np.array_equal(got[i, 1:], g)
        # the oracle
        f_ref, g_ref = J.nll_grad(m_o, cats, jmap, value, th)
        labs, scale = 0.0, np.zeros(joint.n_joint)
        for c, e in enumerate(cats):
            if e["t"].size == 0:
                continue
            thc = J.category_thetas(jmap, value, th)[c]
            logl = (F.nll_grad_terms(m_o, e, thc) if m_o.kind == "phis" else O.nll_grad_terms(m_o, e, thc))[0]
            labs += math.fsum(np.abs(logl))
            sc = _scale(O, F, m_o, e, thc)
            for p in range(jm.shape[1]):
                if jm[c, p] >= 0:
                    scale[jm[c, p]] += sc[p]
        G.assert_nll_grad_close(got[i], f_ref, g_ref, scale, labs)
    return got


TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])


def _map_4d(n_cat):
    """Gamma, sigma, the P-wave amplitudes shared (joint 0..5), F_S and delta_S
    per category (6 .. 6 + 2 n_cat), mu and f_b constants per category."""
    jmap, value = [], []
    for c in range(n_cat):
        jmap.append([0, 1, -1, -1, 2, 3, 4, 5, 6 + c, 6 + n_cat + c])
        value.append([0, 0, 0.002 * c, 0.08 + 0.02 * c, 0, 0, 0, 0, 0, 0])
    return jmap, value


def _theta_4d(n_cat, shift=0.0):
    return np.concatenate([[0.66 + shift, 0.045, 0.52, 0.25 - shift, 3.2, 3.1],
                           0.05 + 0.03 * np.arange(n_cat), 0.3 - 0.4 * np.arange(n_cat) + shift])


def test_joint_4d_parity_and_fixed_order_sum(env):
    O, J, F, G, torch, api = env
    n_cat = 4
    sizes = [[1500, 0, 4097, 513], [2048, 700, 1, 3000]]
    cats = [[synth.events_4d(n, 40 + 10 * i + c, weighted=True) for c, n in enumerate(s)]
            for i, s in enumerate(sizes)]
    jmap, value = _map_4d(n_cat)
    _check_parity(env, O.Model("4d", 0.0, 15.0), api.model_4d(0.0, 15.0), cats, jmap, value,
                  [_theta_4d(n_cat), _theta_4d(n_cat, 0.05)])


def _map_phis(n_bins, omega=0.0):
    """Example 2's categories: bin b, flavour q -> category 2 b + (q < 0).
    Joint: 0 Gamma, 1 A0sq, 2 Apesq, 3 delta_pa, 4 delta_pe, 5 DG, 6 Dm, 7 phi_s,
    then F_S and delta_S of each bin; sigma, mu, f_b, omega, C_SP and the tag
    selector are constants."""
    jmap, value = [], []
    for b in range(n_bins):
        for q in (1.0, -1.0):
            jmap.append([0, -1, -1, -1, 1, 2, 3, 4, 8 + b, 8 + n_bins + b, 5, 6, 7, -1, -1, -1])
            value.append([0, 0.045, 0.0, 0.05, 0, 0, 0, 0, 0, 0, 0, 0, 0, omega, CSP[b], q])
    return jmap, value


def _theta_phis(n_bins):
    return np.concatenate([[0.66, 0.52, 0.25, 3.2, 3.1, 0.085, 17.77, 0.8],
                           0.02 + 0.015 * np.arange(n_bins), 1.2 - 0.5 * np.arange(n_bins)])


def test_joint_phis_twelve_categories_parity(env):
    O, J, F, G, torch, api = env
    n_bins = 6
    jmap, value = _map_phis(n_bins)
    cats = []
    for c in range(2 * n_bins):
        e = synth.events_phis(900 + 137 * c, 70 + c, weighted=True)
        e["q"] = np.full(e["t"].size, value[c][15])
        cats.append(e)
    got = _check_parity(env, O.Model("phis", 0.0, 15.0), api.model_phis(0.0, 15.0), [cats], jmap, value,
                        [_theta_phis(n_bins)])
    assert np.all(np.isfinite(got))


def test_joint_fit_4d_matches_oracle_and_batch_equals_solo(env):
    O, J, F, G, torch, api = env
    n_cat = 4
    m_o, m_g = O.Model("4d", 0.0, 15.0), api.model_4d(0.0, 15.0)
    jmap, value = _map_4d(n_cat)
    truth = _theta_4d(n_cat)
    fits = []
    for i in range(2):
        cats = []
        for c in range(n_cat):
            thc = J.category_thetas(jmap, value, truth)[c]
            cats.append(O.toygen(m_o, thc, 300 + 10 * i + c, [2500], [int(2500 * thc[3] / (1 - thc[3]))])[0])
        fits.append(cats)
    nj = len(truth)
    # limits inside the physical region (A0sq + Apesq < 1, F_S > 0)
    lo = np.array([0.3, 0.01, 0.35, 0.1, 0.0, 0.0] + [1e-3] * n_cat + [-3.2] * n_cat)
    hi = np.array([1.5, 0.2, 0.6, 0.35, 6.3, 6.3] + [0.5] * n_cat + [3.2] * n_cat)
    free = [0, 2, 3, 4, 5] + list(range(6, nj))
    params = [api.Param(float(truth[j]), float(lo[j]), float(hi[j]), float((hi[j] - lo[j]) / 50), fixed=j not in free)
              for j in range(nj)]

    def run(sel):
        cols, off = _pack([fits[i] for i in sel])
        theta = torch.tensor(np.tile(truth, (len(sel), 1)), device="cuda")
        r = api.ipa_fit_joint(m_g, G.to_dev(cols), torch.tensor(off, device="cuda"), api.Joint(jmap, value),
                              params, theta, max_iter=300, tol=1e-9)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in r.items()}

    batch = run([0, 1])
    solo = run([1])
    for key in ("theta", "err", "nll", "status", "iters", "passes"):
        assert np.array_equal(solo[key][0], batch[key][1]), key
    ref = J.fit(m_o, fits[0], jmap, value, truth, free, lo=lo, hi=hi, tol=1e-10)
    assert ref.status == "CONVERGED" and batch["status"][0] in (0, 2)
    for j in free:
        assert abs(batch["theta"][0, j] - ref.theta[j]) < 1e-6 * ref.err[j], (j, batch["theta"][0, j], ref.theta[j])
        assert batch["err"][0, j] == pytest.approx(ref.err[j], rel=1e-3)
    assert batch["nll"][0] == pytest.approx(ref.nll, rel=1e-12)
    # HESSE of both joint fits at their minima: covariance and correlations
    # against the inverse of the oracle's finite-difference Hessian
    cols, off = _pack(fits)
    hs = api.ipa_hesse_joint(m_g, G.to_dev(cols), torch.tensor(off, device="cuda"), api.Joint(jmap, value), params,
                             torch.tensor(batch["theta"], device="cuda"))
    hs = {k: v.cpu().numpy() for k, v in hs.items()}
    assert list(hs["status"]) == [0, 0]
    cov_ref = np.linalg.inv(ref.hess)
    got = hs["cov"][0][np.ix_(free, free)]
    sd = np.sqrt(np.diag(cov_ref))
    np.testing.assert_allclose(got / np.outer(sd, sd), cov_ref / np.outer(sd, sd), atol=2e-3)
    np.testing.assert_allclose(hs["err"][0][free], sd, rtol=1e-3)
    fixed = [j for j in range(nj) if j not in free]
    assert np.all(hs["cov"][0][fixed] == 0.0) and np.all(hs["err"][0][fixed] == 0.0)
    np.testing.assert_allclose(np.diag(hs["corr"][0])[free], 1.0, rtol=1e-12)


def test_joint_minos_matches_the_oracle_profile(env):
    """Three 1D categories: Gamma shared, f_b per category, sigma and mu
    constants.  GPU HESSE and MINOS of Gamma and one f_b at the oracle's joint
    minimum against the oracle's profile-likelihood roots."""
    O, J, F, G, torch, api = env
    m_o, m_g = O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0)
    jmap = [[0, -1, -1, 1], [0, -1, -1, 2], [0, -1, -1, 3]]
    value = [[0.0, 0.045, 0.0, 0.0], [0.0, 0.05, 0.01, 0.0], [0.0, 0.04, -0.01, 0.0]]
    truth = np.array([0.66, 0.1, 0.2, 0.05])
    cats = []
    for c in range(3):
        thc = J.category_thetas(jmap, value, truth)[c]
        n_b = int(4000 * thc[3] / (1 - thc[3]))
        cats.append({"t": O.toygen(m_o, thc, 900 + c, [4000], [n_b])[0]["t"]})
    lo, hi = np.array([0.2, 0.0, 0.0, 0.0]), np.array([2.0, 0.6, 0.6, 0.6])
    params = [api.Param(float(truth[j]), float(lo[j]), float(hi[j]), 0.01) for j in range(4)]
    joint = api.Joint(jmap, value)
    cols, off = _pack([cats])
    ev, offd = G.to_dev(cols), torch.tensor(off, device="cuda")
    # both sides start from the oracle's minimum (the GPU reads the NLL there itself)
    ref = J.fit(m_o, cats, jmap, value, truth, [0, 1, 2, 3], lo=lo, hi=hi, tol=1e-12)
    assert ref.status == "CONVERGED"
    th = torch.tensor(ref.theta[None, :], device="cuda")
    nll = api.ipa_nll_grad_joint(m_g, ev, offd, joint, th)[:, 0].contiguous()
    hs = api.ipa_hesse_joint(m_g, ev, offd, joint, params, th)
    scan = [0, 2]
    mn = api.ipa_minos_joint(m_g, ev, offd, joint, params, th, nll, hs["cov"], scan)
    mn = {k: v.cpu().numpy()[0] for k, v in mn.items()}
    err = np.sqrt(np.diag(np.linalg.inv(ref.hess)))
    for j in scan:
        (elo, ehi), st = J.minos(m_o, cats, jmap, value, ref.theta, ref.nll, [0, 1, 2, 3], j, float(err[j]),
                                 lo=lo, hi=hi)
        assert st == ("OK", "OK") and tuple(mn["status"][j]) == (0, 0), (j, mn["status"][j])
        assert abs(mn["lo"][j] - elo) < 1e-5 * err[j], (j, mn["lo"][j], elo)
        assert abs(mn["hi"][j] - ehi) < 1e-5 * err[j], (j, mn["hi"][j], ehi)
    assert tuple(mn["status"][1]) == (5, 5)          # not scanned


def _sample_one_tag(F, m, th, q, n, seed):
    """Events of one flavour from the model normalised over that tag, by
    accept-reject (uniform t and angles; the bound is 1.5 x the largest density
    of 1e5 candidates, checked against every candidate)."""
    rng = np.random.default_rng(seed)

    def cand(k):
        return {"t": rng.uniform(m.t_lo, m.t_hi, k), "ck": rng.uniform(-1, 1, k), "cl": rng.uniform(-1, 1, k),
                "phi": rng.uniform(-math.pi, math.pi, k), "q": np.full(k, q)}

    bound = 1.5 * F.pdf(m, cand(100000), th).max()
    out = {k: [] for k in ("t", "ck", "cl", "phi", "q")}
    got = 0
    while got < n:
        c = cand(100000)
        p = F.pdf(m, c, th)
        assert p.max() < bound
        keep = rng.uniform(0, bound, p.size) < p
        for k in out:
            out[k].append(c[k][keep])
        got += int(keep.sum())
    return {k: np.concatenate(v)[:n] for k, v in out.items()}


def test_joint_fit_phis_one_flavour_categories_matches_oracle(env):
    """Three m(KK) bins times two flavours; Dm held; the physics parameters
    and each bin's F_S and delta_S free (13 free joint parameters)."""
    O, J, F, G, torch, api = env
    n_bins = 3
    m_o, m_g = O.Model("phis", 0.0, 15.0), api.model_phis(0.0, 15.0)
    jmap, value = _map_phis(n_bins, omega=0.0)
    truth = _theta_phis(n_bins)
    ths = J.category_thetas(jmap, value, truth)
    cats = [_sample_one_tag(F, m_o, ths[c], value[c][15], 1500, 500 + c) for c in range(2 * n_bins)]
    nj = len(truth)
    lo = np.array([0.3, 0.35, 0.1, 0.0, 0.0, -0.5, 10.0, -3.1] + [1e-3] * n_bins + [-3.2] * n_bins)
    hi = np.array([1.5, 0.6, 0.35, 6.3, 6.3, 0.5, 25.0, 3.1] + [0.5] * n_bins + [3.2] * n_bins)
    free = [j for j in range(nj) if j != 6]
    params = [api.Param(float(truth[j]), float(lo[j]), float(hi[j]), float((hi[j] - lo[j]) / 50), fixed=j not in free)
              for j in range(nj)]
    cols, off = _pack([cats])
    theta = torch.tensor(truth[None, :], device="cuda")
    r = api.ipa_fit_joint(m_g, G.to_dev(cols), torch.tensor(off, device="cuda"), api.Joint(jmap, value), params,
                          theta, max_iter=300, tol=1e-9)
    r = {k: v.cpu().numpy() for k, v in r.items()}
    ref = J.fit(m_o, cats, jmap, value, truth, free, lo=lo, hi=hi, tol=1e-10)
    assert ref.status == "CONVERGED" and r["status"][0] in (0, 2)
    for j in free:
        assert abs(r["theta"][0, j] - ref.theta[j]) < 1e-6 * ref.err[j], (j, r["theta"][0, j], ref.theta[j])
        assert r["err"][0, j] == pytest.approx(ref.err[j], rel=1e-3)
    assert r["nll"][0] == pytest.approx(ref.nll, rel=1e-12)


def test_joint_fit_with_32_parameters_and_an_empty_fit(env):
    """The largest joint fit (IPA_MAX_PAR = 32 parameters: Gamma shared, f_b in
    each of 31 1D categories, all free) against the oracle; a second fit whose
    categories are all empty ends IPA_FIT_EMPTY and leaves the first bitwise
    as it is alone."""
    O, J, F, G, torch, api = env
    m_o, m_g = O.Model("1d", 0.3, 15.0), api.model_1d(0.3, 15.0)
    n_cat = 31
    jmap = [[0, -1, -1, 1 + c] for c in range(n_cat)]
    value = [[0.0, 0.045, 0.0, 0.0] for _ in range(n_cat)]
    truth = np.concatenate([[0.66], 0.05 + 0.01 * np.arange(n_cat)])
    cats = []
    for c in range(n_cat):
        thc = J.category_thetas(jmap, value, truth)[c]
        cats.append({"t": O.toygen(m_o, thc, 1200 + c, [1500], [int(1500 * thc[3] / (1 - thc[3]))])[0]["t"]})
    empty = [{"t": np.zeros(0)} for _ in range(n_cat)]
    lo, hi = np.concatenate([[0.2], np.zeros(n_cat)]), np.concatenate([[2.0], np.full(n_cat, 0.8)])
    params = [api.Param(float(truth[j]), float(lo[j]), float(hi[j]), 0.01) for j in range(32)]
    joint = api.Joint(jmap, value)

    def run(fits):
        cols, off = _pack(fits)
        theta = torch.tensor(np.tile(truth, (len(fits), 1)), device="cuda")
        r = api.ipa_fit_joint(m_g, G.to_dev(cols), torch.tensor(off, device="cuda"), joint, params, theta,
                              max_iter=400, tol=1e-9)
        return {k: v.cpu().numpy() for k, v in r.items()}

    both = run([cats, empty])
    solo = run([cats])
    assert both["status"][1] == 4                       # IPA_FIT_EMPTY
    for key in ("theta", "err", "nll", "status", "iters", "passes"):
        assert np.array_equal(both[key][0], solo[key][0]), key
    ref = J.fit(m_o, cats, jmap, value, truth, list(range(32)), lo=lo, hi=hi, tol=1e-10)
    assert ref.status == "CONVERGED" and solo["status"][0] in (0, 2)
    for j in range(32):
        assert abs(solo["theta"][0, j] - ref.theta[j]) < 1e-6 * ref.err[j], (j, solo["theta"][0, j], ref.theta[j])
        assert solo["err"][0, j] == pytest.approx(ref.err[j], rel=1e-3)
