"""Plain FP64 CPU oracle of the flavour-tagged decay-time model with B_s
oscillation and Gaussian resolution (test infrastructure only, like the rest
of ``oracle/``: only tests, the smoke check and the bench's CPU legs use it).

The method (arXiv:1706.01420):

* Sec. 4 (Example 2): the time-dependent fit of B_s and anti-B_s decays (two
  flavour categories) with the physics parameters Delta m_s, Gamma and
  Delta Gamma, and the CP-violating phase;
* Sec. 2 (Software) and "Combining with symbolic programming": the Faddeeva
  function w(z) for the resolution-convolved oscillation terms and their limit
  at large t / sigma.

Reading (the paper prints no formula): the flavour-tagged decay rate of a
CP-even final state with |lambda| = 1,

    S(t, q) = e^{-Gamma t} [cosh(DG t/2) - cos(phi_s) sinh(DG t/2)
                            + q (1 - 2 omega) sin(phi_s) sin(Dm t)],   t >= 0,

for tag q = +1 / -1 with mistag probability omega, convolved with a Gaussian
of width sigma and offset mu.  With Gamma_H = Gamma - DG/2 and Gamma_L = Gamma
+ DG/2 it is a sum of convolved exponentials,

    S = (1 - c)/2 g(tau; Gamma_H) + (1 + c)/2 g(tau; Gamma_L)
        + q D s Im g(tau; Gamma - i Dm),          c = cos phi_s, s = sin phi_s,
                                                  D = 1 - 2 omega, tau = t - mu,

where g(tau; z) = int_0^inf e^{-z u} G(tau - u; sigma) du for complex z.  The
normalisation over t in [t_lo, t_hi] and q = +-1 is N = (1 - c) I_T(Gamma_H) +
(1 + c) I_T(Gamma_L) (the tagged term is odd in q), and with a flat background
P(t, q) = (1 - f_b) S / N + f_b / (2 (t_hi - t_lo)).

Parameters (ABI order): (Gamma, sigma, mu, f_b, DG, Dm, phi_s, omega).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import wofz

from .ipa_oracle import SQRT2, Model, _philox_call, gauss, time_norm_grad, u01

NPAR = 8
IDX = {"Gamma": 0, "sigma": 1, "mu": 2, "f_b": 3, "DG": 4, "Dm": 5, "phi_s": 6, "omega": 7}


def conv_c(tau, z, sigma):
    """g(tau; z) = int_0^inf e^{-z u} G(tau - u; sigma) du for complex z,
    = 1/2 exp(-z tau + z^2 sigma^2 / 2) erfc(u),  u = (z sigma^2 - tau)/(sqrt2 sigma),
    written with the Faddeeva function w(x) = e^{-x^2} erfc(-i x) so that no
    factor over- or underflows: erfc(u) = e^{-u^2} w(i u) for Re u >= 0 and
    erfc(u) = 2 - e^{-u^2} w(-i u) otherwise, with
    exp(-z tau + z^2 sigma^2/2 - u^2) = exp(-tau^2 / (2 sigma^2))."""
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    z = complex(z)
    u = (z * sigma * sigma - tau) / (SQRT2 * sigma)
    gx = np.exp(-tau * tau / (2.0 * sigma * sigma))
    out = np.empty(tau.shape, dtype=complex)
    pos = u.real >= 0.0
    out[pos] = 0.5 * gx[pos] * wofz(1j * u[pos])
    neg = ~pos
    out[neg] = np.exp(-z * tau[neg] + 0.5 * z * z * sigma * sigma) - 0.5 * gx[neg] * wofz(-1j * u[neg])
    return out


def conv_c_grad(tau, z, sigma):
    """(g, dg/dz, dg/dsigma, dg/dtau) for complex z, from differentiating the
    closed form: dg/dz = (z sigma^2 - tau) g - sigma^2 G, dg/dsigma =
    z^2 sigma g - (z sigma + tau/sigma) G, dg/dtau = -z g + G (G the Gaussian)."""
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    g = conv_c(tau, z, sigma)
    G = gauss(tau, sigma)
    return (g, (z * sigma * sigma - tau) * g - sigma * sigma * G,
            z * z * sigma * g - (z * sigma + tau / sigma) * G, -z * g + G)


def _parts(theta):
    Gamma, sigma, mu, f_b, DG, Dm, phi, om = (float(v) for v in theta)
    return Gamma, sigma, mu, f_b, DG, Dm, phi, om, Gamma - 0.5 * DG, Gamma + 0.5 * DG


def norm_grad(model: Model, theta):
    """N and dN/dtheta (8 entries) for N = (1 - c) I_T(Gamma_H) + (1 + c) I_T(Gamma_L)."""
    Gamma, sigma, mu, f_b, DG, Dm, phi, om, GH, GL = _parts(theta)
    c, s = math.cos(phi), math.sin(phi)
    IH = time_norm_grad(GH, sigma, mu, model.t_lo, model.t_hi)   # (I, dGamma, dsigma, dmu)
    IL = time_norm_grad(GL, sigma, mu, model.t_lo, model.t_hi)
    N = (1 - c) * IH[0] + (1 + c) * IL[0]
    d = np.zeros(NPAR)
    d[0] = (1 - c) * IH[1] + (1 + c) * IL[1]
    d[1] = (1 - c) * IH[2] + (1 + c) * IL[2]
    d[2] = (1 - c) * IH[3] + (1 + c) * IL[3]
    d[4] = -0.5 * (1 - c) * IH[1] + 0.5 * (1 + c) * IL[1]
    d[6] = s * IH[0] - s * IL[0]
    return N, d


def signal(model: Model, ev: dict, theta):
    """Unnormalised S(t, q) and dS/dtheta (8 rows; the f_b row is zero)."""
    Gamma, sigma, mu, f_b, DG, Dm, phi, om, GH, GL = _parts(theta)
    t = np.asarray(ev["t"], dtype=np.float64)
    q = np.asarray(ev["q"], dtype=np.float64)
    c, s, D = math.cos(phi), math.sin(phi), 1.0 - 2.0 * om
    tau = t - mu
    gH, dH_G, dH_s, dH_t = (np.real(v) for v in conv_c_grad(tau, GH, sigma))
    gL, dL_G, dL_s, dL_t = (np.real(v) for v in conv_c_grad(tau, GL, sigma))
    gc, dc_z, dc_s, dc_t = conv_c_grad(tau, complex(Gamma, -Dm), sigma)
    aH, aL, Ds = 0.5 * (1 - c), 0.5 * (1 + c), D * s
    S = aH * gH + aL * gL + q * Ds * gc.imag
    dS = np.zeros((NPAR, t.size))
    dS[0] = aH * dH_G + aL * dL_G + q * Ds * dc_z.imag
    dS[1] = aH * dH_s + aL * dL_s + q * Ds * dc_s.imag
    dS[2] = -(aH * dH_t + aL * dL_t + q * Ds * dc_t.imag)
    dS[4] = -0.5 * aH * dH_G + 0.5 * aL * dL_G
    dS[5] = -q * Ds * dc_z.real            # dz/dDm = -i:  Im(-i dg/dz) = -Re(dg/dz)
    dS[6] = 0.5 * s * gH - 0.5 * s * gL + q * D * c * gc.imag
    dS[7] = -2.0 * q * s * gc.imag
    return S, dS


def pdf(model: Model, ev: dict, theta) -> np.ndarray:
    N, _ = norm_grad(model, theta)
    S, _ = signal(model, ev, theta)
    f_b = float(theta[3])
    return (1.0 - f_b) * S / N + f_b / (2.0 * (model.t_hi - model.t_lo))


def nll_grad_terms(model: Model, ev: dict, theta):
    """Per-event w log P and -w (dP/dtheta_j) / P (an (8, N) array)."""
    theta = np.asarray(theta, dtype=np.float64)
    f_b = float(theta[3])
    t = np.asarray(ev["t"], dtype=np.float64)
    w = ev.get("w")
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    N, dN = norm_grad(model, theta)
    S, dS = signal(model, ev, theta)
    V2 = 2.0 * (model.t_hi - model.t_lo)
    P = (1.0 - f_b) * S / N + f_b / V2
    dP = (1.0 - f_b) * (dS / N - np.outer(dN, S) / (N * N))
    dP[3] = -S / N + 1.0 / V2
    return w * np.log(P), -w * dP / P


def nll(model: Model, ev: dict, theta) -> float:
    logl, _ = nll_grad_terms(model, ev, theta)
    return -math.fsum(logl)


def nll_grad(model: Model, ev: dict, theta):
    logl, terms = nll_grad_terms(model, ev, theta)
    return -math.fsum(logl), np.array([math.fsum(row) for row in terms])


def envelope(model: Model, theta) -> float:
    """M_S >= max S(t, q) on the range: |g(tau; z)| <= g(tau; Re z) <= min(1,
    exp(-Re z tau + (Re z)^2 sigma^2 / 2)), so M_S = (1 - c)/2 M(Gamma_H) +
    (1 + c)/2 M(Gamma_L) + |D s| M(Gamma) with M(x) that bound at tau = t_lo - mu."""
    Gamma, sigma, mu, f_b, DG, Dm, phi, om, GH, GL = _parts(theta)

    def M(x):
        return min(1.0, math.exp(-x * (model.t_lo - mu) + 0.5 * x * x * sigma * sigma))

    c, s, D = math.cos(phi), math.sin(phi), 1.0 - 2.0 * om
    return 0.5 * (1 - c) * M(GH) + 0.5 * (1 + c) * M(GL) + abs(D * s) * M(Gamma)


def toy_one(model: Model, theta, seed: int, toy: int, n_sig: int, n_bkg: int, chunk: int = 1 << 16) -> dict:
    """One tagged pseudo-experiment (Sec. 7 accept-reject with counters):
    signal candidate j of toy k draws Philox calls (j_lo, j_hi, k, c):
      c = 0: t = t_lo + u (t_hi - t_lo), u_acc;   c = 1: u_q, unused;
    with q = +1 if u_q <= 1/2 else -1, kept iff u_acc M_S < S(t - mu, q); the toy
    takes the first n_sig kept candidates in increasing j.  Background event i
    uses (i_lo, i_hi, k, 4): t = t_lo + u (t_hi - t_lo) and q from the second
    uniform in the same way."""
    theta = np.asarray(theta, dtype=np.float64)
    span = model.t_hi - model.t_lo
    MS = envelope(model, theta)
    ts, qs = [], []
    got, j0 = 0, 0
    while got < n_sig:
        j = np.arange(j0, j0 + chunk, dtype=np.uint64)
        x = _philox_call(j, toy, 0, seed)
        y = _philox_call(j, toy, 1, seed)
        t = model.t_lo + u01(x[0], x[1]) * span
        q = np.where(u01(y[0], y[1]) <= 0.5, 1.0, -1.0)
        S, _ = signal(model, {"t": t, "q": q}, theta)
        keep = u01(x[2], x[3]) * MS < S
        idx = np.nonzero(keep)[0][: n_sig - got]
        ts.append(t[idx])
        qs.append(q[idx])
        got += idx.size
        j0 += chunk
    if n_bkg > 0:
        i = np.arange(n_bkg, dtype=np.uint64)
        x = _philox_call(i, toy, 4, seed)
        ts.append(model.t_lo + u01(x[0], x[1]) * span)
        qs.append(np.where(u01(x[2], x[3]) <= 0.5, 1.0, -1.0))
    return {"t": np.concatenate(ts) if ts else np.zeros(0), "q": np.concatenate(qs) if qs else np.zeros(0)}
