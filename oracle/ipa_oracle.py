"""Plain, slow, FP64 CPU oracle for the unbinned-likelihood hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / ``--impl reference`` leg of ``bench.py`` may import this module.
The library itself never does: it fails loudly if its CUDA extension is
missing.  Nothing here is shared with the CUDA sources, and nothing here
imports them.

Every function evaluates the plain definition with numpy float64 and
``scipy.special.erfc``; sums are ``math.fsum`` (correctly rounded).  No
blocking, fusion or reassociation beyond the formula as written.

The method (Ipanema-beta, arXiv:1706.01420):

* Sec. 3 (Example 1): unbinned maximum-likelihood fit; per-event PDF, its
  analytic normalisation, the log of the signal/background mixture, and the
  sum of log-likelihoods; FCN = -log L (errors at Delta(-log L) = 1/2).
* Sec. 4 (Example 2): the time-dependent angular fit of Bs -> J/psi K K with
  a P wave (three polarisations) and an S wave; parameters with limits.
* Sec. 7 (Example 5): toy generation by accept-reject with a counter-based
  generator, event counts drawn on the host with Poisson fluctuations.
* Section "Combining with symbolic programming": the angular functions, their
  integrals and derivatives of the Bs -> J/psi K K model.

The paper prints no PDF formula.  The readings used here (all listed in the
design notes with their pins) are:

* time PDF  g(tau) = int_0^inf exp(-Gamma s) G(tau - s; sigma) ds
           = 1/2 exp(-Gamma tau + Gamma^2 sigma^2 / 2) erfc((Gamma sigma^2 - tau)/(sqrt2 sigma)),
  tau = t - mu (exponential decay convolved with a Gaussian resolution);
* angular PDF A(Omega) = sum_k h_k f_k(cos thK, cos thmu, phi), the t = 0,
  no-oscillation helicity-basis form with 10 P/S-wave terms;
* P = (1 - f_b) [g / I_T] [A / I_Omega] + f_b / V on the box
  t in [t_lo, t_hi], cos in [-1, 1], phi in [-pi, pi].

Parameter vectors (index order is the ABI order):
  1D: (Gamma, sigma, mu, f_b)
  4D: (Gamma, sigma, mu, f_b, A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S)
with |A_pa|^2 = 1 - A0sq - Apesq and the P-wave fractions scaled by 1 - F_S.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erfc

SQRT2 = math.sqrt(2.0)
SQRT2PI = math.sqrt(2.0 * math.pi)
I_OMEGA = 16.0 * math.pi / 9.0   # integral of A over the angles when sum |A_i|^2 = 1

IDX = {"Gamma": 0, "sigma": 1, "mu": 2, "f_b": 3, "A0sq": 4, "Apesq": 5,
       "delta_pa": 6, "delta_pe": 7, "F_S": 8, "delta_S": 9}
NPAR = {"1d": 4, "4d": 10, "tag": 8, "phis": 14}


@dataclass
class Model:
    kind: str            # "1d", "4d", "tag" (flavour-tagged decay time, oracle/tagged.py) or
                         # "phis" (time-dependent angular model with tagging, oracle/phis.py)
    t_lo: float
    t_hi: float

    @property
    def npar(self) -> int:
        return NPAR[self.kind]

    @property
    def volume(self) -> float:
        """Volume of the observable box (background density is 1/V)."""
        dt = self.t_hi - self.t_lo
        if self.kind == "tag":
            return 2.0 * dt              # decay time x tag q = +-1
        if self.kind == "phis":
            return 2.0 * dt * 2.0 * 2.0 * 2.0 * math.pi   # decay time x angles x tag
        return dt if self.kind == "1d" else dt * 2.0 * 2.0 * 2.0 * math.pi


# --------------------------------------------------------------------------
# Decay time: exponential convolved with a Gaussian (Sec. 3 normalisation,
# Sec. 4 time distribution)
# --------------------------------------------------------------------------

def gauss(tau, sigma):
    """Unit-area Gaussian density G(tau; sigma)."""
    return np.exp(-0.5 * (tau / sigma) ** 2) / (SQRT2PI * sigma)


def time_conv(tau, Gamma, sigma):
    """g(tau) = int_0^inf exp(-Gamma s) G(tau - s; sigma) ds, closed form."""
    tau = np.asarray(tau, dtype=np.float64)
    z = (Gamma * sigma * sigma - tau) / (SQRT2 * sigma)
    return 0.5 * np.exp(-Gamma * tau + 0.5 * Gamma * Gamma * sigma * sigma) * erfc(z)


def time_conv_grad(tau, Gamma, sigma):
    """(g, dg/dGamma, dg/dsigma, dg/dtau) from differentiating the closed form.

    dg/dtau = -Gamma g + G, dg/dGamma = (Gamma sigma^2 - tau) g - sigma^2 G,
    dg/dsigma = Gamma^2 sigma g - (Gamma sigma + tau / sigma) G.
    """
    tau = np.asarray(tau, dtype=np.float64)
    g = time_conv(tau, Gamma, sigma)
    G = gauss(tau, sigma)
    dg_dtau = -Gamma * g + G
    dg_dG = (Gamma * sigma * sigma - tau) * g - sigma * sigma * G
    dg_ds = Gamma * Gamma * sigma * g - (Gamma * sigma + tau / sigma) * G
    return g, dg_dG, dg_ds, dg_dtau


def normal_cdf(x):
    return 0.5 * erfc(-np.asarray(x, dtype=np.float64) / SQRT2)


def time_antiderivative(tau, Gamma, sigma):
    """F(tau) with dF/dtau = g(tau):  F = [Phi(tau/sigma) - g(tau)] / Gamma."""
    return (normal_cdf(tau / sigma) - time_conv(tau, Gamma, sigma)) / Gamma


def time_norm(Gamma, sigma, mu, t_lo, t_hi):
    """I_T = int_{t_lo}^{t_hi} g(t - mu) dt (analytic normalisation, Sec. 3)."""
    return float(time_antiderivative(t_hi - mu, Gamma, sigma)
                 - time_antiderivative(t_lo - mu, Gamma, sigma))


def time_norm_grad(Gamma, sigma, mu, t_lo, t_hi):
    """(I_T, dI_T/dGamma, dI_T/dsigma, dI_T/dmu).

    dF/dGamma = -(F + dg/dGamma) / Gamma, dF/dsigma = (-(tau/sigma) G - dg/dsigma) / Gamma,
    dF/dmu = -g(tau).
    """
    out = np.zeros(4)
    for sgn, t in ((1.0, t_hi), (-1.0, t_lo)):
        tau = t - mu
        F = float(time_antiderivative(tau, Gamma, sigma))
        g, dg_dG, dg_ds, _ = (float(v) for v in time_conv_grad(tau, Gamma, sigma))
        G = float(gauss(tau, sigma))
        out[0] += sgn * F
        out[1] += sgn * (-(F + dg_dG) / Gamma)
        out[2] += sgn * ((-(tau / sigma) * G - dg_ds) / Gamma)
        out[3] += sgn * (-g)
    return out


# --------------------------------------------------------------------------
# Angular part: 10-term P/S-wave helicity amplitude sum (Sec. 4 and the
# symbolic-programming section: angular functions, integrals, derivatives)
# --------------------------------------------------------------------------

def angular_basis(ck, cl, phi):
    """f_k(cos thK, cos thmu, phi), k = 1..10, as a (10, N) array."""
    ck = np.asarray(ck, dtype=np.float64)
    cl = np.asarray(cl, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    sk = np.sqrt(1.0 - ck * ck)
    sl = np.sqrt(1.0 - cl * cl)
    cp, sp = np.cos(phi), np.sin(phi)
    return np.stack([
        ck * ck * sl * sl,
        0.5 * sk * sk * (1.0 - sl * sl * cp * cp),
        0.5 * sk * sk * (1.0 - sl * sl * sp * sp),
        sk * sk * sl * sl * sp * cp,
        SQRT2 * sk * ck * sl * cl * cp,
        -SQRT2 * sk * ck * sl * cl * sp,
        sl * sl / 3.0,
        (2.0 / math.sqrt(6.0)) * sk * sl * cl * cp,
        -(2.0 / math.sqrt(6.0)) * sk * sl * cl * sp,
        (2.0 / math.sqrt(3.0)) * ck * sl * sl,
    ])


# max |f_k| over the angular box (envelope of the accept-reject generator)
ANGULAR_MAX = np.array([1.0, 0.5, 0.5, 0.5, SQRT2 / 4.0, SQRT2 / 4.0, 1.0 / 3.0,
                        1.0 / math.sqrt(6.0), 1.0 / math.sqrt(6.0), 2.0 / math.sqrt(3.0)])


def amplitude_coeffs(theta):
    """h_k from (A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S); delta_0 = 0."""
    x0, xe, dpa, dpe, F, dS = (float(theta[i]) for i in range(4, 10))
    xa = 1.0 - x0 - xe
    s = 1.0 - F
    a0, apa, ape, aS = math.sqrt(s * x0), math.sqrt(s * xa), math.sqrt(s * xe), math.sqrt(F)
    return np.array([
        a0 * a0, apa * apa, ape * ape,
        apa * ape * math.sin(dpe - dpa),
        a0 * apa * math.cos(dpa),
        a0 * ape * math.sin(dpe),
        aS * aS,
        aS * apa * math.cos(dpa - dS),
        aS * ape * math.sin(dpe - dS),
        aS * a0 * math.cos(dS),
    ])


def amplitude_coeffs_grad(theta):
    """dh_k / dtheta_j for the six angular parameters, shape (10, 6).

    Columns: A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S.  The magnitudes are
    sqrt of products of (1 - F_S) x_i and F_S, differentiated with
    d sqrt(u) = du / (2 sqrt(u)); |A_pa|^2 = 1 - A0sq - Apesq.
    """
    x0, xe, dpa, dpe, F, dS = (float(theta[i]) for i in range(4, 10))
    xa = 1.0 - x0 - xe
    s = 1.0 - F
    r0, ra, re = math.sqrt(x0), math.sqrt(xa), math.sqrt(xe)
    rF, rs = math.sqrt(F), math.sqrt(s)
    c4, c5, c6 = math.sin(dpe - dpa), math.cos(dpa), math.sin(dpe)
    c8, c9, c10 = math.cos(dpa - dS), math.sin(dpe - dS), math.cos(dS)
    d = np.zeros((10, 6))
    # d/dA0sq  (dxa = -1)
    d[:, 0] = [s, -s, 0.0,
               s * (-xe) / (2.0 * ra * re) * c4,
               s * (xa - x0) / (2.0 * r0 * ra) * c5,
               s * xe / (2.0 * r0 * re) * c6,
               0.0,
               rF * rs * (-1.0) / (2.0 * ra) * c8,
               0.0,
               rF * rs / (2.0 * r0) * c10]
    # d/dApesq (dxa = -1)
    d[:, 1] = [0.0, -s, s,
               s * (xa - xe) / (2.0 * ra * re) * c4,
               s * (-x0) / (2.0 * r0 * ra) * c5,
               s * x0 / (2.0 * r0 * re) * c6,
               0.0,
               rF * rs * (-1.0) / (2.0 * ra) * c8,
               rF * rs / (2.0 * re) * c9,
               0.0]
    # d/ddelta_pa
    d[:, 2] = [0.0, 0.0, 0.0,
               -s * ra * re * math.cos(dpe - dpa),
               -s * r0 * ra * math.sin(dpa),
               0.0, 0.0,
               -rF * rs * ra * math.sin(dpa - dS),
               0.0, 0.0]
    # d/ddelta_pe
    d[:, 3] = [0.0, 0.0, 0.0,
               s * ra * re * math.cos(dpe - dpa),
               0.0,
               s * r0 * re * math.cos(dpe),
               0.0, 0.0,
               rF * rs * re * math.cos(dpe - dS),
               0.0]
    # d/dF_S  (ds = -1; d sqrt(F s) = (1 - 2F) / (2 sqrt(F s)))
    dFs = (1.0 - 2.0 * F) / (2.0 * rF * rs)
    d[:, 4] = [-x0, -xa, -xe,
               -ra * re * c4,
               -r0 * ra * c5,
               -r0 * re * c6,
               1.0,
               dFs * ra * c8,
               dFs * re * c9,
               dFs * r0 * c10]
    # d/ddelta_S
    d[:, 5] = [0.0] * 7 + [
        rF * rs * ra * math.sin(dpa - dS),
        -rF * rs * re * math.cos(dpe - dS),
        -rF * rs * r0 * math.sin(dS)]
    return d


# --------------------------------------------------------------------------
# Per-event PDF, NLL and gradient (Sec. 3: log of the mixture, sum of logs)
# --------------------------------------------------------------------------

def _cols(model: Model, ev: dict):
    t = np.asarray(ev["t"], dtype=np.float64)
    w = ev.get("w")
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    return t, w


def pdf(model: Model, ev: dict, theta) -> np.ndarray:
    """Normalised per-event density P(t[, Omega])."""
    if model.kind == "tag":
        from . import tagged
        return tagged.pdf(model, ev, theta)
    if model.kind == "phis":
        from . import phis
        return phis.pdf(model, ev, theta)
    theta = np.asarray(theta, dtype=np.float64)
    Gamma, sigma, mu, f_b = theta[:4]
    t, _ = _cols(model, ev)
    IT = time_norm(Gamma, sigma, mu, model.t_lo, model.t_hi)
    T = time_conv(t - mu, Gamma, sigma)
    if model.kind == "1d":
        sig = T / IT
    else:
        A = amplitude_coeffs(theta) @ angular_basis(ev["ck"], ev["cl"], ev["phi"])
        sig = (T / IT) * (A / I_OMEGA)
    return (1.0 - f_b) * sig + f_b / model.volume


def nll(model: Model, ev: dict, theta) -> float:
    """NLL = -sum_e w_e log P_e, summed with math.fsum."""
    _, w = _cols(model, ev)
    return -math.fsum(w * np.log(pdf(model, ev, theta)))


def nll_grad_terms(model: Model, ev: dict, theta):
    """Per-event terms: (w log P, and -w (dP/dtheta_j) / P as an (npar, N) array)."""
    if model.kind == "tag":
        from . import tagged
        return tagged.nll_grad_terms(model, ev, theta)
    if model.kind == "phis":
        from . import phis
        return phis.nll_grad_terms(model, ev, theta)
    theta = np.asarray(theta, dtype=np.float64)
    Gamma, sigma, mu, f_b = theta[:4]
    t, w = _cols(model, ev)
    V = model.volume
    IT, dIT_G, dIT_s, dIT_mu = time_norm_grad(Gamma, sigma, mu, model.t_lo, model.t_hi)
    T, dT_G, dT_s, dT_tau = time_conv_grad(t - mu, Gamma, sigma)
    dT_mu = -dT_tau
    if model.kind == "1d":
        A = np.ones_like(t)
        IO = 1.0
    else:
        f = angular_basis(ev["ck"], ev["cl"], ev["phi"])
        A = amplitude_coeffs(theta) @ f
        dA = amplitude_coeffs_grad(theta).T @ f       # (6, N)
        IO = I_OMEGA
    S = (T / IT) * (A / IO)                            # normalised signal density
    P = (1.0 - f_b) * S + f_b / V
    dP = np.zeros((model.npar, t.size))
    # time parameters: d(T/IT) = dT/IT - T dIT/IT^2
    for j, dT, dI in ((0, dT_G, dIT_G), (1, dT_s, dIT_s), (2, dT_mu, dIT_mu)):
        dP[j] = (1.0 - f_b) * (A / IO) * (dT / IT - T * dI / (IT * IT))
    dP[3] = -S + 1.0 / V
    if model.kind == "4d":
        dP[4:10] = (1.0 - f_b) * (T / IT) * (dA / IO)
    return w * np.log(P), -w * dP / P


def nll_grad(model: Model, ev: dict, theta):
    """(NLL, dNLL/dtheta) with dNLL/dtheta_j = -sum_e w_e (dP_e/dtheta_j) / P_e."""
    logl, terms = nll_grad_terms(model, ev, theta)
    return -math.fsum(logl), np.array([math.fsum(row) for row in terms])


# --------------------------------------------------------------------------
# Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and toy generation
# (Sec. 7: counter-based generator, accept-reject, host-drawn event counts)
# --------------------------------------------------------------------------

_M32 = np.uint64(0xFFFFFFFF)
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds on uint32 counters (arrays) with a 64-bit key.

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 64-bit
    products), then c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is
    bumped by the Weyl constants (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _M32 for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _M32
    k1 = np.asarray(k1, dtype=np.uint64) & _M32
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _M32
            k1 = (k1 + np.uint64(PHILOX_W1)) & _M32
        p0 = m0 * c0
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _M32,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _M32)
    return c0, c1, c2, c3


def u01(a, b):
    """Two uint32 -> uniform double in (0, 1]: (((a<<32)|b) >> 11) + 1) * 2^-53 (exact)."""
    v = ((np.asarray(a, dtype=np.uint64) << np.uint64(32)) | np.asarray(b, dtype=np.uint64)) >> np.uint64(11)
    return (v + np.uint64(1)).astype(np.float64) * (2.0 ** -53)


def _philox_call(idx, toy, call, seed):
    idx = np.asarray(idx, dtype=np.uint64)
    n = idx.size
    return philox4x32_10(idx & _M32, idx >> np.uint64(32), np.full(n, toy, np.uint64),
                         np.full(n, call, np.uint64), seed & 0xFFFFFFFF, seed >> 32)


def time_envelope(model: Model, theta) -> float:
    """M_T >= max g(t - mu) on the range: g <= 1 and g <= exp(-Gamma tau + Gamma^2 sigma^2 / 2)."""
    Gamma, sigma, mu = float(theta[0]), float(theta[1]), float(theta[2])
    return min(1.0, math.exp(-Gamma * (model.t_lo - mu) + 0.5 * Gamma * Gamma * sigma * sigma))


def angular_envelope(theta) -> float:
    """M_Omega = sum_k |h_k| max|f_k| >= max A(Omega)."""
    return float(np.sum(np.abs(amplitude_coeffs(theta)) * ANGULAR_MAX))


def toy_one(model: Model, theta, seed: int, toy: int, n_sig: int, n_bkg: int,
            chunk: int = 1 << 16) -> dict:
    if model.kind == "tag":
        from . import tagged
        return tagged.toy_one(model, theta, seed, toy, n_sig, n_bkg, chunk)
    return _toy_one_angular(model, theta, seed, toy, n_sig, n_bkg, chunk)


def _toy_one_angular(model: Model, theta, seed: int, toy: int, n_sig: int, n_bkg: int,
                     chunk: int = 1 << 16) -> dict:
    """One pseudo-experiment: n_sig accepted signal candidates then n_bkg background events.

    Signal candidate j of toy k draws Philox calls counter (j_lo, j_hi, k, c), c = 0,1,2:
      c=0: t = t_lo + u*(t_hi - t_lo), u_t;   c=1: ck = 2u - 1, cl = 2u - 1;
      c=2: phi = pi*(2u - 1), u_a.
    It is kept iff u_t * M_T < g(t - mu) and (4D) u_a * M_Omega < A(Omega); the toy
    takes the first n_sig kept candidates in increasing j.  Background event i
    uses counters (i_lo, i_hi, k, 4) and (.., 5): t, ck, then cl, phi.
    The 1D model uses only the time draws.
    """
    theta = np.asarray(theta, dtype=np.float64)
    Gamma, sigma, mu = theta[0], theta[1], theta[2]
    span = model.t_hi - model.t_lo
    MT = time_envelope(model, theta)
    four = model.kind == "4d"
    if four:
        h = amplitude_coeffs(theta)
        MO = angular_envelope(theta)
    cols = {k: [] for k in (("t", "ck", "cl", "phi") if four else ("t",))}
    got, j0 = 0, 0
    while got < n_sig:
        j = np.arange(j0, j0 + chunk, dtype=np.uint64)
        x = _philox_call(j, toy, 0, seed)
        t = model.t_lo + u01(x[0], x[1]) * span
        keep = u01(x[2], x[3]) * MT < time_conv(t - mu, Gamma, sigma)
        if four:
            y = _philox_call(j, toy, 1, seed)
            z = _philox_call(j, toy, 2, seed)
            ck = 2.0 * u01(y[0], y[1]) - 1.0
            cl = 2.0 * u01(y[2], y[3]) - 1.0
            phi = math.pi * (2.0 * u01(z[0], z[1]) - 1.0)
            A = h @ angular_basis(ck, cl, phi)
            keep &= u01(z[2], z[3]) * MO < A
        idx = np.nonzero(keep)[0][: n_sig - got]
        cols["t"].append(t[idx])
        if four:
            cols["ck"].append(ck[idx]); cols["cl"].append(cl[idx]); cols["phi"].append(phi[idx])
        got += idx.size
        j0 += chunk
    if n_bkg > 0:
        i = np.arange(n_bkg, dtype=np.uint64)
        x = _philox_call(i, toy, 4, seed)
        cols["t"].append(model.t_lo + u01(x[0], x[1]) * span)
        if four:
            y = _philox_call(i, toy, 5, seed)
            cols["ck"].append(2.0 * u01(x[2], x[3]) - 1.0)
            cols["cl"].append(2.0 * u01(y[0], y[1]) - 1.0)
            cols["phi"].append(math.pi * (2.0 * u01(y[2], y[3]) - 1.0))
    return {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in cols.items()}


def toygen(model: Model, theta, seed: int, n_sig, n_bkg, toys=None) -> list[dict]:
    """Pseudo-experiments for the listed toy indices (all by default)."""
    toys = range(len(n_sig)) if toys is None else toys
    return [toy_one(model, theta, seed, k, int(n_sig[k]), int(n_bkg[k])) for k in toys]


# --------------------------------------------------------------------------
# Fit (Sec. 3 / 4: MIGRAD minimisation and HESSE errors, here a plain Newton
# iteration on the analytic gradient with a finite-difference Hessian)
# --------------------------------------------------------------------------

@dataclass
class FitResult:
    theta: np.ndarray
    err: np.ndarray
    nll: float
    status: str
    iterations: int
    hess: np.ndarray = field(repr=False, default=None)


def hessian_fd(model: Model, ev: dict, theta, free, rel=1e-4):
    """Central finite difference of the analytic gradient over the free parameters."""
    return hessian_fd_function(lambda th: nll_grad(model, ev, th), theta, free, rel)


def hessian_fd_function(fn, theta, free, rel=1e-4):
    """The same for any function fn(theta) -> (value, gradient)."""
    theta = np.asarray(theta, dtype=np.float64)
    free = list(free)
    H = np.zeros((len(free), len(free)))
    for a, j in enumerate(free):
        h = rel * max(abs(theta[j]), 1e-2)
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        gp = fn(tp)[1][free]
        gm = fn(tm)[1][free]
        H[:, a] = (gp - gm) / (2.0 * h)
    return 0.5 * (H + H.T)


def fit(model: Model, ev: dict, theta0, free, lo=None, hi=None,
        tol=1e-10, max_iter=100) -> FitResult:
    """Minimise the NLL over the free parameters by damped Newton steps
    (``fit_function`` applied to the model's NLL and gradient)."""
    return fit_function(lambda th: nll_grad(model, ev, th), model.npar, theta0, free, lo=lo, hi=hi, tol=tol,
                        max_iter=max_iter)


def fit_function(fn, n, theta0, free, lo=None, hi=None, tol=1e-10, max_iter=100) -> FitResult:
    """Minimise fn(theta) -> (value, gradient) over the free parameters by damped
    Newton steps.

    Stops when the Newton decrement sqrt(g^T H^-1 g) (the step length in units
    of the parameter errors) is below ``tol``.  Errors are sqrt(diag(H^-1)),
    i.e. Delta NLL = 1/2 (Sec. 3).
    """
    theta = np.asarray(theta0, dtype=np.float64).copy()
    free = list(free)
    lo = np.full(n, -np.inf) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.full(n, np.inf) if hi is None else np.asarray(hi, dtype=np.float64)
    f, g = fn(theta)
    status = "MAXITER"
    it = 0
    for it in range(1, max_iter + 1):
        H = hessian_fd_function(fn, theta, free)
        gf = g[free]
        # modified Newton: shift an indefinite Hessian until it is positive definite
        lam_min, lam_max = np.linalg.eigvalsh(H)[[0, -1]]
        definite = lam_min > 1e-12 * abs(lam_max)
        Hm = H if definite else H + (abs(lam_min) + 1e-6 * abs(lam_max)) * np.eye(len(free))
        step = -np.linalg.solve(Hm, gf)
        dec = math.sqrt(max(0.0, -float(gf @ step)))
        if definite and dec < tol:
            status = "CONVERGED"
            break
        lam = 1.0
        while lam > 1e-6:
            trial = theta.copy()
            trial[free] = np.clip(theta[free] + lam * step, lo[free], hi[free])
            ft, gt = fn(trial)
            if ft <= f:
                break
            lam *= 0.5
        if ft > f:
            status = "CONVERGED" if (definite and dec < 1e-6) else "LINESEARCH"
            break
        theta, f, g = trial, ft, gt
    H = hessian_fd_function(fn, theta, free)
    cov = np.linalg.inv(H)
    err = np.zeros(n)
    err[free] = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return FitResult(theta, err, f, status, it, H)
