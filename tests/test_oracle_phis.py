"""Pins of the oracle's full time-dependent angular model with tagging
(oracle/phis.py).

* Without resolution (sigma = 1e-7) the rate equals a direct construction: the
  amplitudes evolved in time with g+- written out as complex exponentials,
  A_i(t) = A_i [g+ + eta_i lambda g-] (B_s) or A_i [g- + eta_i lambda g+]
  (anti-B_s), put into the muon-helicity sum of Wigner d-functions (the
  independent construction that pins the 4D angular model), mixed by the
  mistag.  A wrong sign, eta, conjugate or product in any of the ten terms
  breaks this equality.
* The PDF integrates to 1 over t, the angles and both tags, or over the one
  tag a category selects; the two one-tag normalisations add up to the
  both-tag one; the complex time integral behind them equals quadrature.
* A pure CP-even (CP-odd) P wave integrated over the angles is the tagged
  decay-time model at phi_s (phi_s + pi); omega = 1/2 makes it tag-blind.
* The gradient equals fourth-order central differences of the NLL.
"""
import cmath
import math

import numpy as np
import pytest
from scipy import integrate

from tests.test_oracle_angular import d1

S2 = math.sqrt(2.0)
TH = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3, 0.085, 17.77, 0.8, 0.3, 0.8, 0.0])


@pytest.fixture(scope="module")
def F():
    from oracle import phis
    return phis


def helicity_rate(thK, thL, phi, A):
    """sum over the muon helicity of |M|^2 for transversity amplitudes A (complex)."""
    A0, Apa, Ape, AS = A
    H = {0: A0, 1: -(Apa + Ape) / S2, -1: -(Apa - Ape) / S2}
    tot = 0.0
    for lam_mu in (1, -1):
        M = sum(H[l] * d1(l, 0, thK) * d1(l, lam_mu, thL) * cmath.exp(1j * l * phi) for l in (-1, 0, 1))
        M += AS / math.sqrt(3.0) * d1(0, lam_mu, thL)
        tot += abs(M) ** 2
    return tot


def random_theta(rng):
    while True:
        x0, xe = rng.uniform(0.05, 0.9, 2)
        if x0 + xe < 0.95:
            break
    return np.array([rng.uniform(0.4, 1.0), 1e-7, 0.0, 0.1, x0, xe, *rng.uniform(-math.pi, math.pi, 2),
                     rng.uniform(0.01, 0.6), rng.uniform(-math.pi, math.pi), rng.uniform(-0.3, 0.3),
                     rng.uniform(0.5, 25.0), rng.uniform(-math.pi, math.pi), rng.uniform(0.0, 0.5), 1.0, 0.0])


def test_matches_time_evolved_helicity_amplitudes(oracle, F):
    rng = np.random.default_rng(7)
    m = oracle.Model("phis", 0.0, 15.0)
    for _ in range(12):
        th = random_theta(rng)
        n = 30
        thK, thL, ph = rng.uniform(0, math.pi, n), rng.uniform(0, math.pi, n), rng.uniform(-math.pi, math.pi, n)
        t = rng.uniform(0.5, 10.0, n)
        q = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0)
        ev = {"t": t, "ck": np.cos(thK), "cl": np.cos(thL), "phi": ph, "q": q}
        got = F.rate(m, ev, th)
        Gamma, DG, Dm, phis, om = th[0], th[10], th[11], th[12], th[13]
        GL, GH = Gamma + DG / 2, Gamma - DG / 2
        A, _ = F.amplitudes(th)
        lam = cmath.exp(-1j * phis)
        ref = []
        for k in range(n):
            eL = cmath.exp(-GL * t[k] / 2)                      # m_L = 0
            eH = cmath.exp(-1j * Dm * t[k] - GH * t[k] / 2)     # m_H = Dm
            gp, gm = (eL + eH) / 2, (eL - eH) / 2
            AB = [A[i] * (gp + F.ETA[i] * lam * gm) for i in range(4)]
            Abar = [A[i] * (gm + F.ETA[i] * lam * gp) for i in range(4)]
            RB = helicity_rate(thK[k], thL[k], ph[k], AB)
            Rb = helicity_rate(thK[k], thL[k], ph[k], Abar)
            ref.append((1 - om) * RB + om * Rb if q[k] > 0 else (1 - om) * Rb + om * RB)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-16)


def _angular_grid(n=4, nphi=8):
    x, wx = np.polynomial.legendre.leggauss(n)
    phi = -math.pi + (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
    CK, CL, PH = np.meshgrid(x, x, phi, indexing="ij")
    W = np.einsum("i,j,k->ijk", wx, wx, np.full(nphi, 2 * math.pi / nphi))
    return CK.ravel(), CL.ravel(), PH.ravel(), W.ravel()


TH2 = np.array([1.2, 0.08, 0.02, 0.3, 0.3, 0.4, 1.0, -2.0, 0.2, -1.0, -0.1, 5.0, -2.0, 0.1, 0.5, 0.0])


@pytest.mark.parametrize("Q", [0.0, 1.0, -1.0])
@pytest.mark.parametrize("th", [TH, TH2])
def test_pdf_integrates_to_one(oracle, F, th, Q):
    """Over t, the angles and both tags (Q = 0), or over the selected tag alone
    (Q = +-1: a category of one flavour)."""
    m = oracle.Model("phis", 0.0, 15.0)
    th = th.copy()
    th[15] = Q
    ck, cl, ph, w = _angular_grid()

    def dens(t, q):
        n = ck.size
        ev = {"t": np.full(n, t), "ck": ck, "cl": cl, "phi": ph, "q": np.full(n, q)}
        return float(F.pdf(m, ev, th) @ w)

    tot = 0.0
    for q in ((-1.0, 1.0) if Q == 0.0 else (Q,)):
        tot += integrate.quad(lambda t: dens(t, q), 0.0, 15.0, limit=4000, points=[0.05, 0.2, 1.0, 3.0],
                              epsrel=1e-12)[0]
    assert abs(tot - 1.0) < 1e-9


def test_one_tag_normalisations_add_up(oracle, F):
    """N_+ + N_- = N over both tags, and so do the gradients; the two differ
    (the tag-odd term is not zero at phi_s = 0.8 with Dm = 5)."""
    m = oracle.Model("phis", 0.0, 15.0)
    for th in (TH, TH2):
        parts = []
        for Q in (1.0, -1.0, 0.0):
            tt = th.copy()
            tt[15] = Q
            parts.append(F.norm_grad(m, tt))
        assert parts[0][0] + parts[1][0] == pytest.approx(parts[2][0], rel=1e-14)
        np.testing.assert_allclose(parts[0][1] + parts[1][1], parts[2][1], rtol=1e-12, atol=1e-14)
        assert abs(parts[0][0] - parts[1][0]) > 1e-4 * parts[2][0]


@pytest.mark.parametrize("Dm", [17.77, 0.5])
def test_complex_time_integral_matches_quadrature(oracle, F, Dm):
    """I_c = int g(t - mu; Gamma - i Dm) dt against adaptive quadrature of the
    convolution (both parts); its derivatives against central differences."""
    from oracle import tagged
    Gamma, sigma, mu, lo, hi = 0.66, 0.045, 0.01, 0.0, 15.0
    z = complex(Gamma, -Dm)
    got = F.time_norm_c_grad(z, sigma, mu, lo, hi)
    edges = np.concatenate([[0.0, 0.05, 0.1, 0.2], np.arange(0.25, 15.0, 0.25), [15.0]])
    for part in (np.real, np.imag):
        ref = math.fsum(integrate.quad(lambda t: float(part(tagged.conv_c(t - mu, z, sigma)[0])), a, b,
                                       limit=200, epsrel=1e-12, epsabs=1e-14)[0] for a, b in zip(edges[:-1], edges[1:]))
        assert float(part(got[0])) == pytest.approx(ref, rel=1e-10, abs=1e-14)
    h = 1e-5

    def I(dz=0.0, ds=0.0, dmu=0.0):
        return F.time_norm_c_grad(z + dz, sigma + ds, mu + dmu, lo, hi)[0]

    assert abs((I(dz=h) - I(dz=-h)) / (2 * h) - got[1]) < 1e-8 * max(abs(got[1]), 1e-3)
    assert abs((I(dz=1j * h) - I(dz=-1j * h)) / (2j * h) - got[1]) < 1e-8 * max(abs(got[1]), 1e-3)
    hs = 1e-7
    assert abs((I(ds=hs) - I(ds=-hs)) / (2 * hs) - got[2]) < 1e-6 * max(abs(got[2]), 1e-3)
    assert abs((I(dmu=hs) - I(dmu=-hs)) / (2 * hs) - got[3]) < 1e-6 * max(abs(got[3]), 1e-3)


@pytest.mark.parametrize("cp", ["even", "odd"])
def test_pure_p_wave_is_the_tagged_model(oracle, F, cp):
    from oracle import tagged
    th = TH.copy()
    th[4], th[5], th[8] = (1.0, 0.0, 0.0) if cp == "even" else (0.0, 1.0, 0.0)
    m = oracle.Model("phis", 0.0, 15.0)
    mt = oracle.Model("tag", 0.0, 15.0)
    ck, cl, ph, w = _angular_grid()
    tt = np.array([TH[0], TH[1], TH[2], TH[3], TH[10], TH[11], TH[12] + (0.0 if cp == "even" else math.pi), TH[13]])
    for t in (0.01, 0.3, 1.7, 6.0):
        for q in (-1.0, 1.0):
            n = ck.size
            ev = {"t": np.full(n, t), "ck": ck, "cl": cl, "phi": ph, "q": np.full(n, q)}
            got = float(F.pdf(m, ev, th) @ w)
            ref = float(tagged.pdf(mt, {"t": np.array([t]), "q": np.array([q])}, tt)[0])
            assert got == pytest.approx(ref, rel=1e-12), (cp, t, q)


def test_csp_scales_the_s_p_interference(oracle, F):
    """rate(C_SP) = rate(1) + (C_SP - 1) x (the three S-P interference terms),
    the latter obtained as rate(1) - rate(0); the normalisation does not change."""
    m = oracle.Model("phis", 0.0, 15.0)
    rng = np.random.default_rng(4)
    n = 300
    ev = {"t": rng.uniform(0, 15, n), "ck": rng.uniform(-1, 1, n), "cl": rng.uniform(-1, 1, n),
          "phi": rng.uniform(-math.pi, math.pi, n), "q": np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0)}
    r = {}
    for csp in (0.0, 0.37, 1.0):
        th = TH.copy()
        th[14] = csp
        r[csp] = F.rate(m, ev, th)
        assert F.norm_grad(m, th)[0] == F.norm_grad(m, TH)[0]
    np.testing.assert_allclose(r[0.37], r[0.0] + 0.37 * (r[1.0] - r[0.0]), rtol=1e-12, atol=1e-15)


def test_half_mistag_is_tag_blind(oracle, F):
    th = TH.copy()
    th[13] = 0.5
    m = oracle.Model("phis", 0.0, 15.0)
    rng = np.random.default_rng(3)
    n = 200
    ev = {"t": rng.uniform(0, 15, n), "ck": rng.uniform(-1, 1, n), "cl": rng.uniform(-1, 1, n),
          "phi": rng.uniform(-math.pi, math.pi, n)}
    p1 = F.pdf(m, dict(ev, q=np.ones(n)), th)
    p2 = F.pdf(m, dict(ev, q=-np.ones(n)), th)
    np.testing.assert_array_equal(p1, p2)


def test_gradient_matches_finite_differences(oracle, F):
    m = oracle.Model("phis", 0.0, 15.0)
    rng = np.random.default_rng(2)
    n = 2000
    ev = {"t": rng.exponential(1.5, n), "ck": rng.uniform(-1, 1, n), "cl": rng.uniform(-1, 1, n),
          "phi": rng.uniform(-math.pi, math.pi, n), "q": np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0),
          "w": rng.normal(1.0, 0.2, n)}
    ev["t"] = np.minimum(ev["t"], 14.9)
    base = TH + np.array([0.01, 0.002, 0.001, 0.02, 0.01, -0.01, 0.05, -0.05, 0.01, 0.1, 0.01, 0.05, 0.05, 0.01,
                          0.03, 0.0])
    for Q in (0.0, 1.0, -1.0):
        th = base.copy()
        th[15] = Q
        e = ev if Q == 0.0 else dict(ev, q=np.full(n, Q))
        f, g = F.nll_grad(m, e, th)
        assert g[15] == 0.0

        def nll(d, j):
            tt = th.copy()
            tt[j] += d
            return F.nll(m, e, tt)

        for j in range(15):
            h = 1e-5 * max(abs(th[j]), 1e-2)
            fd = (8 * (nll(h, j) - nll(-h, j)) - (nll(2 * h, j) - nll(-2 * h, j))) / (12 * h)
            assert abs(fd - g[j]) <= 1e-6 * max(abs(g[j]), 1.0), (Q, j, fd, g[j])


@pytest.mark.parametrize("Q", [0.0, 1.0])
def test_envelope_bounds_the_rate(oracle, F, Q):
    """u B_i < rate is a valid accept-reject test only if the bin bound B_i >=
    rate everywhere in bin i: random parameter points (C_SP up to 1.3) against
    2e5 random (t, angles, tag)."""
    m = oracle.Model("phis", 0.0, 15.0)
    rng = np.random.default_rng(11)
    for _ in range(15):
        th = random_theta(rng)
        th[1], th[2], th[14], th[15] = rng.uniform(0.02, 0.08), rng.uniform(-0.02, 0.02), rng.uniform(0, 1.3), Q
        n = 200000
        ev = {"t": np.concatenate([rng.uniform(0, 0.3, n // 2), rng.uniform(0, 15, n // 2)]),
              "ck": rng.uniform(-1, 1, n), "cl": rng.uniform(-1, 1, n), "phi": rng.uniform(-math.pi, math.pi, n),
              "q": np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0)}
        w, edges, B, C = F.envelope_bins(m, th)
        b = np.minimum(((ev["t"] - m.t_lo) / w).astype(np.int64), F.GEN_BINS - 1)
        # points on a bin's boundary belong to both neighbours: take the left one too
        left = np.maximum(b - 1, 0)
        r = F.rate(m, ev, th)
        assert np.all((r <= B[b]) | ((ev["t"] == edges[b]) & (r <= B[left])))
        assert C[0] == 0.0 and all(C[i + 1] == C[i] + B[i] for i in range(F.GEN_BINS))


def test_toys_recover_the_parameters(oracle, F):
    """Exact counts, the selected tag, and a fit of Gamma, phi_s and F_S to a
    one-flavour toy lands within 4.5 sigma of the generating values."""
    m = oracle.Model("phis", 0.0, 15.0)
    th = TH.copy()
    th[13], th[15] = 0.0, -1.0
    toy = F.toy_one(m, th, 77, 3, 12000, 1000)
    assert toy["t"].size == 13000 and np.all(toy["q"] == -1.0)
    assert np.all((toy["t"] >= 0) & (toy["t"] <= 15)) and np.all(np.abs(toy["ck"]) <= 1)
    free = [0, 8, 12]
    r = oracle.fit_function(lambda x: F.nll_grad(m, toy, x), F.NPAR, th, free, tol=1e-8, max_iter=60)
    assert r.status == "CONVERGED"
    for j in free:
        assert abs(r.theta[j] - th[j]) < 4.5 * r.err[j], (j, r.theta[j], th[j], r.err[j])
    toy0 = F.toy_one(m, TH, 78, 0, 500, 20)
    assert set(np.unique(toy0["q"])) == {-1.0, 1.0} and toy0["t"].size == 520
