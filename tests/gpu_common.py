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


def assert_nll_grad_close(got, f_ref, g_ref, scale, logl_abs, rtol_f=1e-12, rtol_g=1e-9):
    f_got, g_got = float(got[0]), np.asarray(got[1:])
    assert abs(f_got - f_ref) <= rtol_f * logl_abs, (f_got, f_ref, (f_got - f_ref) / logl_abs)
    bound = rtol_g * np.maximum(np.abs(g_ref), scale)
    bad = np.abs(g_got - g_ref) > bound
    assert not bad.any(), {"got": g_got[bad], "ref": g_ref[bad], "bound": bound[bad]}
