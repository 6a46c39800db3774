"""Plain FP64 CPU oracle of the full time-dependent angular model of
B_s -> J/psi K K with flavour tagging (test infrastructure only, like the rest
of ``oracle/``: only tests, the smoke check and the bench's CPU legs use it).

The method (arXiv:1706.01420, Sec. 4, Example 2): the phi_s fit of
B_s -> J/psi K K in decay time and the three helicity angles, P wave (three
polarisations) and S wave, with the widths Gamma_L, Gamma_H (the cosh and
sinh terms), the flavour-tagged oscillation Delta m_s and the CP-violating
phase; the resolution-convolved oscillation uses the Faddeeva function
(Sec. 2).  The paper prints no formula; the reading here is the plain time
evolution of the transversity amplitudes:

* amplitudes A_i, i = 0, para, perp, S, as in the 4D model (``ipa_oracle``:
  |A_i|^2 from A0sq, Apesq with the P wave scaled by 1 - F_S, |A_S|^2 = F_S,
  delta_0 = 0), CP eigenvalues eta = (+1, +1, -1, -1);
* a B_s produced at t = 0 decays with A_i(t) = A_i [g+(t) + eta_i lambda g-(t)],
  a anti-B_s with A_i [g-(t) + eta_i lambda g+(t)] (the common factor p/q
  dropped, |q/p| = 1, |lambda| = 1), lambda = e^{-i phi_s},
  g+-(t) = (e^{-i m_L t - Gamma_L t/2} +- e^{-i m_H t - Gamma_H t/2}) / 2,
  Gamma_L,H = Gamma +- DG/2, Dm = m_H - m_L;
* the ten angular terms are the bilinears of the 4D model with A_i -> A_i(t):
  |A_0|^2, |A_pa|^2, |A_pe|^2, Im(A_pa* A_pe), Re(A_0* A_pa), Im(A_0* A_pe),
  |A_S|^2, Re(A_S* A_pa), Im(A_S* A_pe), Re(A_S* A_0), each times f_k(Omega);
* the products of g's are sums of exponentials,
  |g+-|^2 = (E_L + E_H +- 2 E_c) / 4,  g+* g- = (E_L - E_H + 2i E_s) / 4,
  g-* g+ = (E_L - E_H - 2i E_s) / 4,  E_L,H = e^{-Gamma_L,H t},
  E_c + i E_s = e^{-Gamma t} e^{i Dm t};
  with the Gaussian resolution (sigma, offset mu) each becomes its
  convolution: E_L,H -> g(tau; Gamma_L,H), E_c + i E_s -> g(tau; Gamma - i Dm)
  (``tagged.conv_c``);
* tag q = +1 (B_s) or -1, mistag omega: rate(q) = (1 - omega) R_q + omega R_-q;
* normalisation over t in [t_lo, t_hi], the angles and both tags (the
  oscillating terms cancel in the sum over tags and the interference terms in
  the angular integral): N = (16 pi / 9) sum_i |A_i|^2 [(1 + eta_i c) I(Gamma_L)
  + (1 - eta_i c) I(Gamma_H)], c = cos phi_s;
* P = (1 - f_b) rate / N + f_b / (2 (t_hi - t_lo) 8 pi).

* the three S-P interference terms carry a factor C_SP (the overlap of the S-
  and P-wave lineshapes in a m(KK) category; 1 for one category covering the
  whole range).
* a category holding the events of one flavour (Example 2 fits six m(KK) bins
  times the two B flavours, each category with its own integral) is
  normalised over that tag only: selector Q = +1 or -1 (Q = 0: both tags).
  Summed over the angles only the |A_i|^2 terms remain, and their tag-odd
  part is q D eta_i |A_i|^2 sin(phi_s) Im g(tau; Gamma - i Dm), so
  N_Q = N / 2 + Q K D sin(phi_s) (sum_i eta_i |A_i|^2) Im I_c with
  I_c = int g(t - mu; Gamma - i Dm) dt over [t_lo, t_hi] and K = 16 pi / 9;
  the background's volume is halved.  I_c comes from the antiderivative
  (Phi - g) / z of the complex convolution (g' = G - z g).

Parameters (ABI order): Gamma, sigma, mu, f_b, A0sq, Apesq, delta_pa,
delta_pe, F_S, delta_S, DG, Dm, phi_s, omega, C_SP, Q (a selector held fixed:
its gradient component is 0).  Events: t, ck, cl, phi, q.
"""
from __future__ import annotations

import math

import numpy as np

from . import ipa_oracle as O
from . import tagged as T

NPAR = 16
QNORM = 15                  # the tag-normalisation selector
SP_TERMS = (7, 8, 9)       # the S-P interference terms, scaled by C_SP
ETA = (1.0, 1.0, -1.0, -1.0)
# (i, j, part) of the ten bilinears conj(A_i) A_j, part 'r' = Re, 'i' = Im
PAIRS = ((0, 0, "r"), (1, 1, "r"), (2, 2, "r"), (1, 2, "i"), (0, 1, "r"), (0, 2, "i"), (3, 3, "r"),
         (3, 1, "r"), (3, 2, "i"), (3, 0, "r"))
ANG = (4, 5, 6, 7, 8, 9)   # the six amplitude parameters


def amplitudes(theta, grad: bool = True):
    """(A_0, A_pa, A_pe, A_S) and dA/d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S), shape (4, 6)
    (None without grad; the derivatives need every magnitude above zero)."""
    x0, xe, dpa, dpe, F, dS = (float(theta[i]) for i in ANG)
    xa = 1.0 - x0 - xe
    s = 1.0 - F
    e_pa, e_pe, e_S = np.exp(1j * dpa), np.exp(1j * dpe), np.exp(1j * dS)
    r0, ra, re, rF = math.sqrt(s * x0), math.sqrt(s * xa), math.sqrt(s * xe), math.sqrt(F)
    A = np.array([r0, ra * e_pa, re * e_pe, rF * e_S], dtype=complex)
    if not grad:
        return A, None
    dA = np.zeros((4, 6), dtype=complex)
    # d sqrt(s x) / dx = s / (2 sqrt(s x)); d/dF of sqrt(s x) = -x / (2 sqrt(s x)); xa = 1 - x0 - xe
    dA[0, 0] = s / (2.0 * r0)
    dA[1, 0] = -s / (2.0 * ra) * e_pa
    dA[1, 1] = -s / (2.0 * ra) * e_pa
    dA[2, 1] = s / (2.0 * re) * e_pe
    dA[1, 2] = 1j * A[1]
    dA[2, 3] = 1j * A[2]
    dA[0, 4] = -x0 / (2.0 * r0)
    dA[1, 4] = -xa / (2.0 * ra) * e_pa
    dA[2, 4] = -xe / (2.0 * re) * e_pe
    dA[3, 4] = 1.0 / (2.0 * rF) * e_S
    dA[3, 5] = 1j * A[3]
    return A, dA


def _products(gL, gH, gc):
    """|g+|^2, |g-|^2, g+* g-, g-* g+ (convolved)."""
    PP = 0.25 * (gL + gH + 2.0 * gc.real)
    MM = 0.25 * (gL + gH - 2.0 * gc.real)
    PM = 0.25 * (gL - gH + 2j * gc.imag)
    MP = 0.25 * (gL - gH - 2j * gc.imag)
    return PP, MM, PM, MP


def _observed(b, ei, ej, lam, q, om, PP, MM, PM, MP):
    """(1 - omega) R_q + omega R_-q of the bilinear conj(A_i(t)) A_j(t) with b = conj(A_i) A_j."""
    X = b * (PP + ej * lam * PM + ei * np.conj(lam) * MP + ei * ej * MM)     # B_s at t = 0
    Y = b * (MM + ej * lam * MP + ei * np.conj(lam) * PM + ei * ej * PP)     # anti-B_s at t = 0
    Rq = np.where(q > 0, X, Y)
    Rm = np.where(q > 0, Y, X)
    return (1.0 - om) * Rq + om * Rm, X, Y


def _part(z, p):
    return z.real if p == "r" else z.imag


def rate(model: O.Model, ev: dict, theta):
    """Unnormalised rate(t, Omega, q) (each event's own tag)."""
    return rate_grad(model, ev, theta, grad=False)[0]


def rate_grad(model: O.Model, ev: dict, theta, grad: bool = True):
    """rate and d rate / d theta (16 rows; the f_b and selector rows are zero; None without grad)."""
    theta = np.asarray(theta, dtype=np.float64)
    Gamma, sigma, mu = (float(theta[i]) for i in range(3))
    DG, Dm, phi, om = (float(theta[i]) for i in range(10, 14))
    GL, GH = Gamma + 0.5 * DG, Gamma - 0.5 * DG
    z = complex(Gamma, -Dm)
    t = np.asarray(ev["t"], dtype=np.float64)
    q = np.asarray(ev["q"], dtype=np.float64)
    tau = t - mu
    f = O.angular_basis(ev["ck"], ev["cl"], ev["phi"])
    cL = T.conv_c_grad(tau, GL, sigma)       # (g, dg/dz, dg/dsigma, dg/dtau)
    cH = T.conv_c_grad(tau, GH, sigma)
    cC = T.conv_c_grad(tau, z, sigma)
    gL, gH = cL[0].real, cH[0].real
    gc = cC[0]
    A, dA = amplitudes(theta, grad)
    lam = complex(math.cos(phi), -math.sin(phi))
    dlam = -1j * lam
    PP, MM, PM, MP = _products(gL, gH, gc)
    n = t.size
    R = np.zeros(n)
    dR = np.zeros((NPAR, n))

    # derivatives of (gL, gH, gc) in the time parameters: Gamma, sigma, mu, DG, Dm
    tg = {
        0: (cL[1].real, cH[1].real, cC[1]),
        1: (cL[2].real, cH[2].real, cC[2]),
        2: (-cL[3].real, -cH[3].real, -cC[3]),
        10: (0.5 * cL[1].real, -0.5 * cH[1].real, 0.0 * cC[1]),
        11: (0.0 * gL, 0.0 * gH, -1j * cC[1]),
    }
    dprod = {j: _products(*v) for j, v in tg.items()}
    csp = float(theta[14])
    for k, (i, j, p) in enumerate(PAIRS):
        b = np.conj(A[i]) * A[j]
        ei, ej = ETA[i], ETA[j]
        Ok, X, Y = _observed(b, ei, ej, lam, q, om, PP, MM, PM, MP)
        if k in SP_TERMS:
            dR[14] += f[k] * _part(Ok, p)
            b = csp * b
            Ok, X, Y = _observed(b, ei, ej, lam, q, om, PP, MM, PM, MP)
        R += f[k] * _part(Ok, p)
        if not grad:
            continue
        # amplitude parameters
        for a in range(6):
            db = np.conj(dA[i, a]) * A[j] + np.conj(A[i]) * dA[j, a]
            if k in SP_TERMS:
                db = csp * db
            if db != 0:
                dO = _observed(db, ei, ej, lam, q, om, PP, MM, PM, MP)[0]
                dR[ANG[a]] += f[k] * _part(dO, p)
        # phi_s: d lambda = -i lambda, d conj(lambda) = conj(d lambda)
        Xd = b * (ej * dlam * PM + ei * np.conj(dlam) * MP)
        Yd = b * (ej * dlam * MP + ei * np.conj(dlam) * PM)
        dO = (1.0 - om) * np.where(q > 0, Xd, Yd) + om * np.where(q > 0, Yd, Xd)
        dR[12] += f[k] * _part(dO, p)
        # omega
        dR[13] += f[k] * _part(np.where(q > 0, Y - X, X - Y), p)
        # time parameters
        for jj, (dPP, dMM, dPM, dMP) in dprod.items():
            dO = _observed(b, ei, ej, lam, q, om, dPP, dMM, dPM, dMP)[0]
            dR[jj] += f[k] * _part(dO, p)
    return R, (dR if grad else None)


def time_norm_c_grad(z, sigma, mu, t_lo, t_hi):
    """(I_c, dI_c/dz, dI_c/dsigma, dI_c/dmu) of I_c = int_{t_lo}^{t_hi} g(t - mu; z) dt for
    complex z, from the antiderivative F = (Phi(tau / sigma) - g(tau; z)) / z and
    dF/dz = -(F + dg/dz) / z, dF/dsigma = (-(tau / sigma) G - dg/dsigma) / z,
    dF/dmu = -g (the real case of ``ipa_oracle.time_norm_grad`` with z complex)."""
    z = complex(z)
    out = np.zeros(4, dtype=complex)
    for sgn, t in ((1.0, t_hi), (-1.0, t_lo)):
        tau = t - mu
        g, dg_dz, dg_ds, _ = (complex(v[0]) for v in T.conv_c_grad(tau, z, sigma))
        G = float(O.gauss(tau, sigma))
        Fv = (float(O.normal_cdf(tau / sigma)) - g) / z
        out[0] += sgn * Fv
        out[1] += sgn * (-(Fv + dg_dz) / z)
        out[2] += sgn * ((-(tau / sigma) * G - dg_ds) / z)
        out[3] += sgn * (-g)
    return out


def _tag_of(theta) -> float:
    """The normalisation's tag: 0 (both tags), +1 or -1 (the sign of the selector)."""
    Q = float(theta[QNORM])
    return 0.0 if Q == 0.0 else math.copysign(1.0, Q)


def norm_grad(model: O.Model, theta):
    """N and dN/dtheta (16 entries): over both tags, or over the selected tag."""
    theta = np.asarray(theta, dtype=np.float64)
    Gamma, sigma, mu = (float(theta[i]) for i in range(3))
    DG, phi = float(theta[10]), float(theta[12])
    GL, GH = Gamma + 0.5 * DG, Gamma - 0.5 * DG
    c, s = math.cos(phi), math.sin(phi)
    IL = O.time_norm_grad(GL, sigma, mu, model.t_lo, model.t_hi)   # (I, dGamma, dsigma, dmu)
    IH = O.time_norm_grad(GH, sigma, mu, model.t_lo, model.t_hi)
    A, _ = amplitudes(theta, grad=False)
    m2 = np.abs(A) ** 2
    # d|A_i|^2 / d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S), from |A_i|^2 = (1 - F) x_i, F
    x0, xe, F = float(theta[4]), float(theta[5]), float(theta[8])
    xa = 1.0 - x0 - xe
    dm2 = np.array([[1 - F, 0, 0, 0, -x0, 0], [-(1 - F), -(1 - F), 0, 0, -xa, 0],
                    [0, 1 - F, 0, 0, -xe, 0], [0, 0, 0, 0, 1.0, 0]])
    eta = np.array(ETA)
    wL, wH = float(np.sum(m2 * (1 + eta * c))), float(np.sum(m2 * (1 - eta * c)))
    K = 16.0 * math.pi / 9.0
    N = K * (wL * IL[0] + wH * IH[0])
    d = np.zeros(NPAR)
    d[0] = K * (wL * IL[1] + wH * IH[1])
    d[1] = K * (wL * IL[2] + wH * IH[2])
    d[2] = K * (wL * IL[3] + wH * IH[3])
    d[10] = K * (0.5 * wL * IL[1] - 0.5 * wH * IH[1])
    for a in range(6):
        dwL = float(np.sum(dm2[:, a] * (1 + eta * c)))
        dwH = float(np.sum(dm2[:, a] * (1 - eta * c)))
        d[ANG[a]] = K * (dwL * IL[0] + dwH * IH[0])
    d[12] = K * (float(np.sum(m2 * (-eta * s))) * IL[0] + float(np.sum(m2 * (eta * s))) * IH[0])
    Q = _tag_of(theta)
    if Q == 0.0:
        return N, d
    # one tag: half the even part plus the tag-odd part Q K D s W Im I_c
    Dm, om = float(theta[11]), float(theta[13])
    D = 1.0 - 2.0 * om
    W = float(np.sum(eta * m2))
    Ic = time_norm_c_grad(complex(Gamma, -Dm), sigma, mu, model.t_lo, model.t_hi)
    odd = K * D * s * W
    N = 0.5 * N + Q * odd * Ic[0].imag
    d = 0.5 * d
    d[0] += Q * odd * Ic[1].imag                 # d/dGamma = d/dz
    d[1] += Q * odd * Ic[2].imag
    d[2] += Q * odd * Ic[3].imag
    d[11] += Q * odd * (-1j * Ic[1]).imag        # d/dDm = -i d/dz
    d[12] += Q * K * D * c * W * Ic[0].imag
    d[13] += Q * K * (-2.0) * s * W * Ic[0].imag
    for a in range(6):
        d[ANG[a]] += Q * K * D * s * float(np.sum(eta * dm2[:, a])) * Ic[0].imag
    return N, d


def volume(model: O.Model, theta=None) -> float:
    """Volume of (t, the angles, the tags) the background is flat over: one tag
    when theta selects one."""
    v = 2.0 * (model.t_hi - model.t_lo) * 8.0 * math.pi
    return v if theta is None or _tag_of(theta) == 0.0 else 0.5 * v


def pdf(model: O.Model, ev: dict, theta) -> np.ndarray:
    N, _ = norm_grad(model, theta)
    R = rate(model, ev, theta)
    f_b = float(theta[3])
    return (1.0 - f_b) * R / N + f_b / volume(model, theta)


def nll_grad_terms(model: O.Model, ev: dict, theta):
    """Per-event w log P and -w (dP/dtheta_j) / P (a (16, N) array)."""
    theta = np.asarray(theta, dtype=np.float64)
    f_b = float(theta[3])
    t = np.asarray(ev["t"], dtype=np.float64)
    w = ev.get("w")
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    N, dN = norm_grad(model, theta)
    R, dR = rate_grad(model, ev, theta)
    V = volume(model, theta)
    P = (1.0 - f_b) * R / N + f_b / V
    dP = (1.0 - f_b) * (dR / N - np.outer(dN, R) / (N * N))
    dP[3] = -R / N + 1.0 / V
    return w * np.log(P), -w * dP / P


def nll(model: O.Model, ev: dict, theta) -> float:
    logl, _ = nll_grad_terms(model, ev, theta)
    return -math.fsum(logl)


def nll_grad(model: O.Model, ev: dict, theta):
    logl, terms = nll_grad_terms(model, ev, theta)
    return -math.fsum(logl), np.array([math.fsum(row) for row in terms])


# --------------------------------------------------------------------------
# Pseudo-experiments (Sec. 7, Example 5: accept-reject with counter-based
# Philox draws), with the model's own envelope
# --------------------------------------------------------------------------

GEN_BINS = 64       # decay-time bins of the generator's envelope


def envelope_bins(model: O.Model, theta):
    """The generator's envelope, piecewise constant in t: (w, edges, B, C) with
    bin width w = (t_hi - t_lo) / 64, left edges e_i = t_lo + i w, bounds
    B_i >= rate(t, Omega, q) for t in bin i, and C the running sums of B
    (C_0 = 0, C_{i+1} = C_i + B_i, in order).  Each observed bilinear is a convex
    mix of b (PP +- ...) terms with |PP|, |MM|, |PM|, |MP| <= (gL + gH + 2 |gc|) / 4
    (|gc| <= g(tau; Gamma)), so |term k| <= |b_k| (gL + gH + 2 |gc|); a convolved
    exponential g(tau; x) decreases in tau and is at most min(1, e^{-x tau +
    x^2 sigma^2 / 2}), taken at the bin's left edge: B_i = (m(Gamma_L) +
    m(Gamma_H) + 2 m(Gamma)) sum_k max|f_k| |b_k| r_k (r_k = |C_SP| for the S-P
    terms, else 1)."""
    theta = np.asarray(theta, dtype=np.float64)
    Gamma, sigma, mu = (float(theta[i]) for i in range(3))
    DG = float(theta[10])
    GL, GH = Gamma + 0.5 * DG, Gamma - 0.5 * DG
    A, _ = amplitudes(theta, grad=False)
    ang = 0.0
    for k, (i, j, _) in enumerate(PAIRS):
        r = abs(float(theta[14])) if k in SP_TERMS else 1.0
        ang += O.ANGULAR_MAX[k] * abs(A[i]) * abs(A[j]) * r
    w = (model.t_hi - model.t_lo) / GEN_BINS
    edges = np.array([model.t_lo + i * w for i in range(GEN_BINS)])

    def m(x, e):
        return min(1.0, math.exp(-x * (e - mu) + 0.5 * x * x * sigma * sigma))

    B = np.array([(m(GL, e) + m(GH, e) + 2.0 * m(Gamma, e)) * ang for e in edges])
    C = np.zeros(GEN_BINS + 1)
    for i in range(GEN_BINS):
        C[i + 1] = C[i] + B[i]
    return w, edges, B, C


def toy_one(model: O.Model, theta, seed: int, toy: int, n_sig: int, n_bkg: int, chunk: int = 1 << 16) -> dict:
    """One pseudo-experiment of the phi_s model (Sec. 7 accept-reject with
    counters, the proposal piecewise uniform in t with the envelope's bin
    bounds as weights).  Signal candidate j of toy k draws Philox calls
    (j_lo, j_hi, k, c):
      c = 0: u_bin, u_acc;   c = 1: ck = 2u - 1, cl = 2u - 1;
      c = 2: phi = pi (2u - 1), u_pos;   c = 3: u_q, unused;
    its bin is the first i with u_bin C_64 <= C_{i+1}, t = min(e_i + u_pos w,
    t_hi); q = the selected tag when the normalisation selector Q is +-1, else
    +1 if u_q <= 1/2 and -1 otherwise; kept iff u_acc B_i < rate(t, Omega, q);
    the toy takes the first n_sig kept candidates in increasing j.  Background
    event i uses (i_lo, i_hi, k, 4): t = t_lo + u (t_hi - t_lo), ck; (.., 5): cl,
    phi; (.., 6): u_q (the tag as for the signal)."""
    theta = np.asarray(theta, dtype=np.float64)
    span = model.t_hi - model.t_lo
    w, edges, B, C = envelope_bins(model, theta)
    Q = _tag_of(theta)

    def tag(u):
        return np.full(u.shape, Q) if Q != 0.0 else np.where(u <= 0.5, 1.0, -1.0)

    cols = {k: [] for k in ("t", "ck", "cl", "phi", "q")}
    got, j0 = 0, 0
    while got < n_sig:
        j = np.arange(j0, j0 + chunk, dtype=np.uint64)
        x = O._philox_call(j, toy, 0, seed)
        y = O._philox_call(j, toy, 1, seed)
        z = O._philox_call(j, toy, 2, seed)
        v = O._philox_call(j, toy, 3, seed)
        b = np.searchsorted(C[1:], O.u01(x[0], x[1]) * C[-1], side="left")
        ev = {"t": np.minimum(edges[b] + O.u01(z[2], z[3]) * w, model.t_hi),
              "ck": 2.0 * O.u01(y[0], y[1]) - 1.0, "cl": 2.0 * O.u01(y[2], y[3]) - 1.0,
              "phi": math.pi * (2.0 * O.u01(z[0], z[1]) - 1.0), "q": tag(O.u01(v[0], v[1]))}
        keep = O.u01(x[2], x[3]) * B[b] < rate(model, ev, theta)
        idx = np.nonzero(keep)[0][: n_sig - got]
        for k in cols:
            cols[k].append(ev[k][idx])
        got += idx.size
        j0 += chunk
    if n_bkg > 0:
        i = np.arange(n_bkg, dtype=np.uint64)
        x = O._philox_call(i, toy, 4, seed)
        y = O._philox_call(i, toy, 5, seed)
        v = O._philox_call(i, toy, 6, seed)
        cols["t"].append(model.t_lo + O.u01(x[0], x[1]) * span)
        cols["ck"].append(2.0 * O.u01(x[2], x[3]) - 1.0)
        cols["cl"].append(2.0 * O.u01(y[0], y[1]) - 1.0)
        cols["phi"].append(math.pi * (2.0 * O.u01(y[2], y[3]) - 1.0))
        cols["q"].append(tag(O.u01(v[0], v[1])))
    return {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in cols.items()}
