"""Pins of the oracle's 10-term angular PDF.

The main pin is an independent construction: A(Omega) must equal the sum over the
muon helicity difference Lambda = +-1 of |M_Lambda|^2, with M_Lambda built from
Wigner small-d functions of the K K (spin 1 and spin 0) and mu mu systems.
Helicity convention of this reading: H_0 = A_0, H_(+-1) = -(A_pa +- A_pe)/sqrt2,
the S wave enters with 1/sqrt(3).  A wrong coefficient, sign or index in any of
the ten terms breaks this equality.  Further pins: the angular integrals by
Gauss-Legendre quadrature, the textbook cos(theta_K) marginal, the bounds
max|f_k| used by the generator, and the coefficient derivatives.
"""
import cmath
import math

import numpy as np
import pytest

S2 = math.sqrt(2.0)


def d1(m, mp, th):
    """Wigner d^1_{m m'}(theta)."""
    c, s = math.cos(th), math.sin(th)
    return {(1, 1): (1 + c) / 2, (1, 0): -s / S2, (1, -1): (1 - c) / 2,
            (0, 1): s / S2, (0, 0): c, (0, -1): -s / S2,
            (-1, 1): (1 - c) / 2, (-1, 0): s / S2, (-1, -1): (1 + c) / 2}[(m, mp)]


def amplitude_sum(thK, thL, phi, theta):
    x0, xe, dpa, dpe, F, dS = theta[4:10]
    xa = 1.0 - x0 - xe
    s = 1.0 - F
    A0 = math.sqrt(s * x0)
    Apa = math.sqrt(s * xa) * cmath.exp(1j * dpa)
    Ape = math.sqrt(s * xe) * cmath.exp(1j * dpe)
    AS = math.sqrt(F) * cmath.exp(1j * dS)
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
    return np.array([0.66, 0.045, 0.0, 0.1, x0, xe, *rng.uniform(-math.pi, math.pi, 2),
                     rng.uniform(0.01, 0.6), rng.uniform(-math.pi, math.pi)])


def test_matches_helicity_amplitude_sum(oracle):
    rng = np.random.default_rng(3)
    for _ in range(40):
        th = random_theta(rng)
        thK = rng.uniform(0, math.pi, 25)
        thL = rng.uniform(0, math.pi, 25)
        phi = rng.uniform(-math.pi, math.pi, 25)
        A = oracle.amplitude_coeffs(th) @ oracle.angular_basis(np.cos(thK), np.cos(thL), phi)
        ref = [amplitude_sum(a, b, c, th) for a, b, c in zip(thK, thL, phi)]
        np.testing.assert_allclose(A, ref, rtol=1e-11, atol=1e-14)


def angular_grid(n=48, nphi=64):
    x, wx = np.polynomial.legendre.leggauss(n)
    phi = -math.pi + (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
    CK, CL, PH = np.meshgrid(x, x, phi, indexing="ij")
    W = np.einsum("i,j,k->ijk", wx, wx, np.full(nphi, 2 * math.pi / nphi))
    return CK.ravel(), CL.ravel(), PH.ravel(), W.ravel()


def test_angular_integrals(oracle):
    ck, cl, phi, w = angular_grid()
    f = oracle.angular_basis(ck, cl, phi)
    got = f @ w
    want = (16 * math.pi / 9) * np.array([1, 1, 1, 0, 0, 0, 1, 0, 0, 0], dtype=float)
    np.testing.assert_allclose(got, want, atol=2e-13)
    assert oracle.I_OMEGA == pytest.approx(16 * math.pi / 9, rel=1e-16)


def test_cos_thetaK_marginal(oracle):
    """Integrating out cos(theta_mu) and phi leaves the textbook polarisation form
    (8 pi / 3) [|A0|^2 c^2 + (|Apa|^2 + |Ape|^2)(1 - c^2) / 2 + |AS|^2 / 3
    + (2/sqrt3) |AS||A0| cos(dS) c]."""
    rng = np.random.default_rng(5)
    th = random_theta(rng)
    x, wx = np.polynomial.legendre.leggauss(40)
    nphi = 48
    phi = -math.pi + (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
    h = oracle.amplitude_coeffs(th)
    for c in (-0.9, -0.3, 0.0, 0.45, 0.8):
        CL, PH = np.meshgrid(x, phi, indexing="ij")
        A = h @ oracle.angular_basis(np.full(CL.size, c), CL.ravel(), PH.ravel())
        marg = float(A @ np.repeat(wx, nphi)) * (2 * math.pi / nphi)
        x0, xe, F, dS = th[4], th[5], th[8], th[9]
        a0sq, apasq, apesq = (1 - F) * x0, (1 - F) * (1 - x0 - xe), (1 - F) * xe
        want = (8 * math.pi / 3) * (a0sq * c * c + 0.5 * (apasq + apesq) * (1 - c * c) + F / 3
                                     + (2 / math.sqrt(3)) * math.sqrt(F * a0sq) * math.cos(dS) * c)
        assert marg == pytest.approx(want, rel=1e-12)


def test_basis_bounds(oracle):
    n = 121
    g = np.linspace(-1, 1, n)
    p = np.linspace(-math.pi, math.pi, 4 * n)
    CK, CL, PH = np.meshgrid(g, g, p, indexing="ij")
    f = oracle.angular_basis(CK.ravel(), CL.ravel(), PH.ravel())
    m = np.abs(f).max(axis=1)
    assert np.all(m <= oracle.ANGULAR_MAX * (1 + 1e-12))
    assert np.all(m >= 0.98 * oracle.ANGULAR_MAX)


def test_pdf_non_negative(oracle):
    rng = np.random.default_rng(11)
    ck, cl, phi = rng.uniform(-1, 1, 20000), rng.uniform(-1, 1, 20000), rng.uniform(-math.pi, math.pi, 20000)
    f = oracle.angular_basis(ck, cl, phi)
    for _ in range(200):
        A = oracle.amplitude_coeffs(random_theta(rng)) @ f
        assert A.min() > -1e-15


def test_coeff_derivatives_vs_finite_differences(oracle):
    rng = np.random.default_rng(7)
    for _ in range(10):
        th = random_theta(rng)
        d = oracle.amplitude_coeffs_grad(th)
        for c, j in enumerate(range(4, 10)):
            h = 1e-6
            tp, tm = th.copy(), th.copy()
            tp[j] += h
            tm[j] -= h
            fd = (oracle.amplitude_coeffs(tp) - oracle.amplitude_coeffs(tm)) / (2 * h)
            np.testing.assert_allclose(d[:, c], fd, rtol=1e-6, atol=1e-8)


def test_full_4d_pdf_integrates_to_one(oracle):
    """Integrate the oracle's 4D density itself: Gauss-Legendre x midpoint grid in the
    angles at each time node, adaptive quadrature in time."""
    from scipy import integrate
    m = oracle.Model("4d", 0.0, 15.0)
    th = np.array([0.66, 0.045, 0.003, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
    ck, cl, phi, w = angular_grid(24, 32)

    def over_angles(t):
        ev = {"t": np.full(ck.size, t), "ck": ck, "cl": cl, "phi": phi}
        return float(oracle.pdf(m, ev, th) @ w)

    total = integrate.quad(over_angles, 0.0, 15.0, points=[0.05, 0.3, 2.0], epsabs=0,
                           epsrel=1e-12, limit=400)[0]
    assert total == pytest.approx(1.0, rel=1e-11)
