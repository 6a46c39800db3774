"""Helpers shared by the GPU parity tests (loaded only when a GPU is present)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_01420_gb300 import build
    build.build()


def to_dev(cols: dict) -> dict:
    return {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda") for k, v in cols.items()}


def grad_scale(O, m, ev, th):
    """Condition scale of each gradient component: the sum over events of the
    absolute values of the pieces the derivative is built from,
    sum_e w_e (|signal-part derivative pieces|) / P_e.  A sum computed in FP64
    in any order is accurate to a small multiple of eps times this scale."""
    th = np.asarray(th, dtype=np.float64)
    Gamma, sigma, mu, f_b = th[:4]
    t = np.asarray(ev["t"])
    w = np.abs(np.asarray(ev["w"])) if ev.get("w") is not None else np.ones_like(t)
    IT, *dIT = O.time_norm_grad(Gamma, sigma, mu, m.t_lo, m.t_hi)
    T, dG, dS, dTau = O.time_conv_grad(t - mu, Gamma, sigma)
    if m.kind == "1d":
        A, IO = np.ones_like(t), 1.0
    else:
        f = O.angular_basis(ev["ck"], ev["cl"], ev["phi"])
        A, IO = O.amplitude_coeffs(th) @ f, O.I_OMEGA
        dh = np.abs(O.amplitude_coeffs_grad(th))
    P = O.pdf(m, ev, th)
    cs = (1 - f_b) / (IT * IO)
    out = np.zeros(m.npar)
    for j, d in enumerate((dG, dS, -dTau)):
        out[j] = cs * math.fsum(w * A * (np.abs(d) + T * abs(dIT[j] / IT)) / P)
    out[3] = math.fsum(w * (T * A / (IT * IO) + 1.0 / m.volume) / P)
    if m.kind == "4d":
        for j in range(6):
            out[4 + j] = cs * math.fsum(w * T * (dh[:, j] @ np.abs(f)) / P)
    return out


def grad_scale_tagged(O, T, m, ev, th):
    """Condition scale of each gradient component: sum over events of |w| / P
    times the absolute values of the pieces the kernel adds for it (each
    derivative of g is a sum of terms in g, tau g and the Gaussian)."""
    Gamma, sigma, mu, f_b, DG, Dm, phi, om = (float(v) for v in th)
    GH, GL = Gamma - DG / 2, Gamma + DG / 2
    c, s, D = math.cos(phi), math.sin(phi), 1 - 2 * om
    aH, aL, Ds = (1 - c) / 2, (1 + c) / 2, D * s
    t = np.asarray(ev["t"])
    w = np.abs(np.asarray(ev["w"])) if ev.get("w") is not None else np.ones_like(t)
    tau = t - mu
    G = O.gauss(tau, sigma)
    gH = np.abs(T.conv_c(tau, GH, sigma))
    gL = np.abs(T.conv_c(tau, GL, sigma))
    z = complex(Gamma, -Dm)
    gc = np.abs(T.conv_c(tau, z, sigma))
    at = np.abs(tau)

    def pieces(x, g):
        ax = abs(x)
        return (ax * sigma ** 2 * g + at * g + sigma ** 2 * G,
                ax * ax * sigma * g + ax * sigma * G + at / sigma * G,
                ax * g + G)

    pH, pL, pC = pieces(GH, gH), pieces(GL, gL), pieces(z, gc)
    N, dN = T.norm_grad(m, th)
    S, _ = T.signal(m, ev, th)
    P = T.pdf(m, ev, th)
    cs = (1 - f_b) / N
    r = w / P
    rows = [aH * pH[0] + aL * pL[0] + abs(Ds) * pC[0],
            aH * pH[1] + aL * pL[1] + abs(Ds) * pC[1],
            aH * pH[2] + aL * pL[2] + abs(Ds) * pC[2],
            None,
            0.5 * aH * pH[0] + 0.5 * aL * pL[0],
            abs(Ds) * pC[0],
            0.5 * abs(s) * (gH + gL) + abs(D * c) * gc,
            2 * abs(s) * gc]
    out = np.zeros(8)
    for j, row in enumerate(rows):
        if row is None:
            out[j] = math.fsum(r * (np.abs(S) / N + 1 / (2 * (m.t_hi - m.t_lo))))
        else:
            out[j] = cs * math.fsum(r * (row + np.abs(S) * abs(dN[j] / N)))
    return out


def assert_nll_grad_close(got, f_ref, g_ref, scale, logl_abs, rtol_f=1e-12, rtol_g=1e-9):
    f_got, g_got = float(got[0]), np.asarray(got[1:])
    assert abs(f_got - f_ref) <= rtol_f * logl_abs, (f_got, f_ref, (f_got - f_ref) / logl_abs)
    bound = rtol_g * np.maximum(np.abs(g_ref), scale)
    bad = np.abs(g_got - g_ref) > bound
    assert not bad.any(), {"got": g_got[bad], "ref": g_ref[bad], "bound": bound[bad]}


def report_margin(name, got, f_ref, g_ref, scale):
    """Print (pytest -s, or -rP) how far inside the tolerances a result is: the
    NLL's relative error, and per gradient component the error relative to |g_j|
    and to the condition scale B_j that the 1e-9 bound uses."""
    got = np.asarray(got)
    g_ref, scale = np.asarray(g_ref), np.asarray(scale)
    d = np.abs(got[1:] - g_ref)
    nz = np.abs(g_ref) > 0
    rel_g = float((d[nz] / np.abs(g_ref[nz])).max()) if nz.any() else 0.0
    rel_b = float((d / np.maximum(np.maximum(np.abs(g_ref), scale), 1e-300)).max())
    print(f"MARGIN {name}: nll rel {abs(float(got[0]) - f_ref) / abs(f_ref):.2e}, "
          f"max |dg|/|g| {rel_g:.2e}, max |dg|/max(|g|,B) {rel_b:.2e}, "
          f"max B/|g| {float((scale[nz] / np.abs(g_ref[nz])).max()) if nz.any() else 0.0:.2e}")
