"""GPU parity at the edges of the likelihood kernel's branches, against the oracle.

Random inputs reach the kernel's rare branches only by chance.  Here events are
placed on them deliberately and compared with the oracle (Eq. of the time PDF
and the helicity sum of Sec. 4) event by event (one event per segment of
ipa_nll_grad_segmented) and tile by tile (segments of 512 events, whole tiles
of the event loop):

* cos(theta_K) or cos(theta_mu) = +-1, +-0 and +-(1 - 2^-17) and its two
  neighbours (the fixed-point angular products hand over to FP64 there);
* phi = +-pi (the double nearest pi), its neighbours and +-0;
* t at both ends of the range and within a few ulps of the cut beyond which
  the Gaussian/erfcx term is dropped (t = mu + Gamma sigma^2 + 6.25 sqrt2 sigma);
* weights 0, negative, 1 and others;
* a steep decay (Gamma = 46.5 ps^-1, no background) whose P reach 1e-302, far
  below the range of the reciprocal's fast path (whole tiles are redone by the
  plain loop);
* parameters outside the model's domain give NaN, and the fitter reports them
  as IPA_FIT_BAD_PDF.

Per event, a gradient component can be built only from angular products that
vanish (sin phi at phi = pi times small sines): there the tolerance adds what
FP64 itself cannot resolve (the change a last-bit step of an input makes) and
the kernel's documented absolute accuracy of the fixed-point angular products
(a few 2^-60, int_math.cuh).
"""
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
TH1 = np.array([0.66, 0.045, 0.0, 0.1])
C17 = 1.0 - 2.0 ** -17
COS_EDGES = [1.0, -1.0, 0.0, -0.0, C17, -C17, np.nextafter(C17, 0.0), np.nextafter(C17, 2.0),
             -np.nextafter(C17, 0.0), -np.nextafter(C17, 2.0)]
PHI_EDGES = [np.pi, -np.pi, np.nextafter(np.pi, 0.0), np.nextafter(-np.pi, 0.0), 0.0, -0.0, np.pi / 2]
WEIGHTS = [0.0, -0.5, 1.0, 2.5, 0.3]


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def t_edges(th, t_lo, t_hi):
    """Range ends and the near-peak cut with its neighbouring doubles."""
    Gamma, sigma, mu = th[0], th[1], th[2]
    cut = mu + (Gamma * sigma * sigma + 6.25 * math.sqrt(2.0) * sigma)
    vals = [t_lo, t_hi, np.nextafter(t_lo, t_hi), np.nextafter(t_hi, t_lo)]
    x = cut
    for _ in range(3):
        x = np.nextafter(x, -np.inf)
    for _ in range(7):
        vals.append(x)
        x = np.nextafter(x, np.inf)
    return vals


def edge_events_4d(th, seed, t_lo=0.0, t_hi=15.0):
    """Random 4D events, each with one or more coordinates on an edge."""
    base = synth.events_4d(400, seed, t_lo=t_lo, t_hi=t_hi)
    rows = []
    i = 0

    def take():
        nonlocal i
        r = {k: base[k][i] for k in ("t", "ck", "cl", "phi")}
        i += 1
        return r

    for c in COS_EDGES:
        r = take(); r["ck"] = c; rows.append(r)
        r = take(); r["cl"] = c; rows.append(r)
        r = take(); r["ck"] = c; r["cl"] = -c; r["phi"] = np.pi; rows.append(r)
    for p in PHI_EDGES:
        r = take(); r["phi"] = p; rows.append(r)
    for t in t_edges(th, t_lo, t_hi):
        r = take(); r["t"] = t; rows.append(r)
        r = take(); r["t"] = t; r["ck"] = 1.0; r["phi"] = -np.pi; rows.append(r)
    return {k: np.array([r[k] for r in rows]) for k in ("t", "ck", "cl", "phi")}


def input_condition(O, m_o, cols, th, terms):
    """Per event and gradient component, the largest change of the oracle's term
    when one input coordinate moves by one ulp: no FP64 evaluation can resolve a
    term more finely than its inputs do (at phi = pi the double's sine is
    1.2e-16 while a one-ulp step of phi moves it by 4.4e-16)."""
    cond = np.zeros_like(terms)
    keys = [k for k in ("t", "ck", "cl", "phi") if k in cols]
    for k in keys:
        for d in (-np.inf, np.inf):
            c2 = dict(cols)
            c2[k] = np.nextafter(cols[k], d)
            if k in ("ck", "cl"):
                c2[k] = np.clip(c2[k], -1.0, 1.0)
            _, t2 = O.nll_grad_terms(m_o, c2, th)
            cond = np.maximum(cond, np.abs(t2 - terms))
    return cond


# The kernel evaluates the angular products f'_k in Q62 fixed point with an
# absolute (not relative) error of a few 2^-60 (int_math.cuh); 2^-57 bounds it.
BASIS_ABS_ERR = 2.0 ** -57


def basis_error(O, m_o, cols, th):
    """Per event and gradient component, the change that an absolute error of
    BASIS_ABS_ERR in every angular product can make to the term: through
    S_k for the six angular parameters (cs w T |dh_kj| / P summed over k),
    through A' for the others (|term| sum_k |h_k| / A)."""
    if m_o.kind != "4d":
        return 0.0
    th = np.asarray(th, dtype=np.float64)
    t = np.asarray(cols["t"])
    w = np.abs(np.asarray(cols["w"])) if cols.get("w") is not None else np.ones_like(t)
    IT = O.time_norm_grad(th[0], th[1], th[2], m_o.t_lo, m_o.t_hi)[0]
    T = O.time_conv_grad(t - th[2], th[0], th[1])[0]
    P = O.pdf(m_o, cols, th)
    f = O.angular_basis(cols["ck"], cols["cl"], cols["phi"])
    h = O.amplitude_coeffs(th)
    A = h @ f
    cs = (1 - th[3]) / (IT * O.I_OMEGA)
    dh = np.abs(O.amplitude_coeffs_grad(th))          # (10, 6)
    _, terms = O.nll_grad_terms(m_o, cols, th)
    err = np.zeros_like(terms)
    for j in range(4):
        err[j] = np.abs(terms[j]) * BASIS_ABS_ERR * np.abs(h).sum() / np.maximum(np.abs(A), 1e-300)
    for j in range(6):
        err[4 + j] = cs * w * T / P * BASIS_ABS_ERR * dh[:, j].sum()
    return err


def per_event_check(O, G, m_o, cols, th, got):
    """Each event's NLL term to 1e-12 and its gradient to 1e-9 of max(|g_j|, B_j)
    (the condition scale of the other parity tests), plus twice the change the
    inputs' own last bit makes to the term, plus what the documented absolute
    accuracy of the fixed-point angular products allows (basis_error)."""
    logl, terms = O.nll_grad_terms(m_o, cols, th)
    cond = input_condition(O, m_o, cols, th, terms) + 2.0 * basis_error(O, m_o, cols, th)
    n = cols["t"].size
    for e in range(n):
        one = {k: v[e:e + 1] for k, v in cols.items()}
        scale = G.grad_scale(O, m_o, one, th)
        f_ref = -float(logl[e])
        assert abs(float(got[e][0]) - f_ref) <= 1e-12 * max(abs(f_ref), 1e-300), (e, got[e][0], f_ref)
        bound = 1e-9 * np.maximum(np.abs(terms[:, e]), scale) + 2.0 * cond[:, e]
        bad = np.abs(got[e][1:] - terms[:, e]) > bound
        assert not bad.any(), {"event": e, "cols": {k: v[e] for k, v in cols.items()},
                               "got": got[e][1:][bad], "ref": terms[bad, e], "bound": bound[bad]}


@pytest.mark.parametrize("weighted", [False, True])
def test_edge_events_one_by_one_4d(env, weighted):
    O, G, torch, api = env
    m, m_o = api.model_4d(0.0, 15.0), O.Model("4d", 0.0, 15.0)
    cols = edge_events_4d(TH4, 5)
    if weighted:
        cols["w"] = np.resize(np.array(WEIGHTS), cols["t"].size)
    n = cols["t"].size
    ev = G.to_dev(cols)
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    got = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(np.tile(TH4, (n, 1)), device="cuda")).cpu().numpy()
    per_event_check(O, G, m_o, cols, TH4, got)
    if weighted:
        zero = np.asarray(cols["w"]) == 0.0
        assert np.all(got[zero] == 0.0)


def scatter_edges(cols, edges, seed):
    """Copy the edge events into random positions of `cols` (in place)."""
    rng = np.random.default_rng(seed)
    n, k = cols["t"].size, edges["t"].size
    pos = rng.choice(n, size=4 * k, replace=False)
    for j, p in enumerate(pos):
        for key in edges:
            cols[key][p] = edges[key][j % k]
    return cols


@pytest.mark.parametrize("weighted", [False, True])
def test_edge_events_in_whole_tiles_4d(env, weighted):
    """Whole 512-event tiles (the software-pipelined event loop) with the edge
    events scattered over lanes and rows, tile sums against the oracle."""
    O, G, torch, api = env
    m, m_o = api.model_4d(0.0, 15.0), O.Model("4d", 0.0, 15.0)
    n_tiles = 24
    cols = synth.events_4d(512 * n_tiles, 17, weighted=weighted)
    edges = edge_events_4d(TH4, 6)
    if weighted:
        edges["w"] = np.resize(np.array(WEIGHTS), edges["t"].size)
    scatter_edges(cols, edges, 18)
    ev = G.to_dev(cols)
    off = torch.arange(0, 512 * n_tiles + 1, 512, dtype=torch.int64, device="cuda")
    got = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(np.tile(TH4, (n_tiles, 1)), device="cuda"))
    got = got.cpu().numpy()
    whole = api.ipa_nll_grad(m, ev, torch.tensor(TH4, device="cuda")).cpu().numpy()
    for s in range(n_tiles):
        c = {k: v[512 * s:512 * (s + 1)] for k, v in cols.items()}
        f_ref, g_ref = O.nll_grad(m_o, c, TH4)
        logl, _ = O.nll_grad_terms(m_o, c, TH4)
        G.assert_nll_grad_close(got[s], f_ref, g_ref, G.grad_scale(O, m_o, c, TH4), math.fsum(np.abs(logl)))
    f_ref, g_ref = O.nll_grad(m_o, cols, TH4)
    logl, _ = O.nll_grad_terms(m_o, cols, TH4)
    G.assert_nll_grad_close(whole, f_ref, g_ref, G.grad_scale(O, m_o, cols, TH4), math.fsum(np.abs(logl)))


@pytest.mark.parametrize("kind", ["1d", "4d"])
def test_tiny_probabilities_steep_decay(env, kind):
    """Gamma = 46.5 (47) ps^-1 and no background: P falls to ~1e-302 at t = 15 ps,
    below the fast reciprocal's range in every tile (each tile is redone by the
    plain loop); tile sums, single events and the whole set against the oracle."""
    O, G, torch, api = env
    th = (TH4 if kind == "4d" else TH1).copy()
    th[0], th[3] = (46.5 if kind == "4d" else 47.0), 0.0
    t_lo, t_hi = 0.0, 15.0
    m = api.model_4d(t_lo, t_hi) if kind == "4d" else api.model_1d(t_lo, t_hi)
    m_o = O.Model(kind, t_lo, t_hi)
    n_tiles = 6
    if kind == "4d":
        cols = synth.events_4d(512 * n_tiles, 21)
    else:
        cols = {"t": synth.events_1d(512 * n_tiles, 21)}
    rng = np.random.default_rng(22)
    far = rng.choice(cols["t"].size, 300, replace=False)
    cols["t"][far] = rng.uniform(14.0, 15.0, far.size)
    cols["t"][far[:8]] = np.array([15.0, t_lo, 14.999999999999998, 10.0, 12.5, 14.9, t_lo + 1e-9, 7.0])
    ev = G.to_dev(cols)
    _, terms = O.nll_grad_terms(m_o, cols, th)
    P = O.pdf(m_o, cols, th)
    assert 1e-307 < P.min() < 1e-300 < P.max()
    off = torch.arange(0, 512 * n_tiles + 1, 512, dtype=torch.int64, device="cuda")
    got = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(np.tile(th, (n_tiles, 1)), device="cuda"))
    got = got.cpu().numpy()
    for s in range(n_tiles):
        c = {k: v[512 * s:512 * (s + 1)] for k, v in cols.items()}
        f_ref, g_ref = O.nll_grad(m_o, c, th)
        logl, _ = O.nll_grad_terms(m_o, c, th)
        G.assert_nll_grad_close(got[s], f_ref, g_ref, G.grad_scale(O, m_o, c, th), math.fsum(np.abs(logl)))
    one = {k: v[far[:8]] for k, v in cols.items()}
    ev1 = G.to_dev(one)
    off1 = torch.arange(9, dtype=torch.int64, device="cuda")
    got1 = api.ipa_nll_grad_segmented(m, ev1, off1, torch.tensor(np.tile(th, (8, 1)), device="cuda"))
    per_event_check(O, G, m_o, one, th, got1.cpu().numpy())


def test_edge_times_1d(env):
    O, G, torch, api = env
    m, m_o = api.model_1d(0.3, 15.0), O.Model("1d", 0.3, 15.0)
    ts = np.array(t_edges(TH1, 0.3, 15.0) + list(synth.events_1d(20, 23)))
    for w in (None, np.resize(np.array(WEIGHTS), ts.size)):
        cols = {"t": ts.copy()} if w is None else {"t": ts.copy(), "w": w}
        ev = G.to_dev(cols)
        n = ts.size
        off = torch.arange(n + 1, dtype=torch.int64, device="cuda")
        got = api.ipa_nll_grad_segmented(m, ev, off, torch.tensor(np.tile(TH1, (n, 1)), device="cuda"))
        per_event_check(O, G, m_o, cols, TH1, got.cpu().numpy())


@pytest.mark.parametrize("kind,index,value", [("4d", 8, 1.5), ("4d", 1, -0.045), ("4d", 3, 1.2), ("4d", 0, -0.5),
                                              ("4d", 4, -0.1), ("1d", 1, -0.045), ("1d", 3, -0.2)])
def test_parameters_outside_the_domain_give_nan(env, kind, index, value):
    O, G, torch, api = env
    th = (TH4 if kind == "4d" else TH1).copy()
    th[index] = value
    if kind == "4d":
        m, cols = api.model_4d(0.0, 15.0), synth.events_4d(3000, 31)
    else:
        m, cols = api.model_1d(0.3, 15.0), {"t": synth.events_1d(3000, 31)}
    ev = G.to_dev(cols)
    out = api.ipa_nll_grad(m, ev, torch.tensor(th, device="cuda")).cpu().numpy()
    assert np.all(np.isnan(out)), out
    assert np.isnan(float(api.ipa_nll(m, ev, torch.tensor(th, device="cuda")).cpu()[0]))


def test_fit_started_outside_the_domain_is_bad_pdf(env):
    O, G, torch, api = env
    m = api.model_4d(0.0, 15.0)
    cols = synth.events_4d(5000, 32)
    ev = G.to_dev(cols)
    lo = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
    hi = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 2.0, 3.2])
    step = np.array([0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2])
    start = TH4.copy()
    start[8] = 1.5
    params = [api.Param(float(start[i]), float(lo[i]), float(hi[i]), float(step[i]), fixed=False) for i in range(10)]
    off = torch.tensor([0, 5000], dtype=torch.int64, device="cuda")
    r = api.ipa_fit_batch(m, ev, off, params, torch.tensor(start[None, :], device="cuda"), max_iter=50, tol=1e-8)
    assert int(r["status"].cpu()[0]) == 3   # IPA_FIT_BAD_PDF
