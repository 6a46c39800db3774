"""Thin Python binding of the C ABI: the same names as include/ipanema.h.

Argument marshalling only: torch CUDA tensors in, device pointers and the
current torch stream out to libipanema.so.  Every step of the likelihood,
generator and fitter runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _capi as C


class IpaError(RuntimeError):
    pass


def _lib():
    return C.load()


def _check(status: int, what: str):
    if status != C.IPA_OK:
        msg = _lib().ipa_last_error().decode(errors="replace")
        raise IpaError(f"{what}: {C.STATUS_NAMES.get(status, status)}: {msg}")


def _ptr(x: torch.Tensor | None, dtype=torch.float64, name="tensor") -> int | None:
    if x is None:
        return None
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise IpaError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise IpaError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise IpaError(f"{name} must be contiguous")
    return x.data_ptr()


def _need(x: torch.Tensor | None, n: int, name: str):
    """Reject a buffer that holds fewer than n elements (the library writes or
    reads n)."""
    if x is not None and x.numel() < n:
        raise IpaError(f"{name} holds {x.numel()} values, the call needs {n}")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def ipa_model_init(kind: int, t_lo: float, t_hi: float) -> C.ipa_model:
    m = C.ipa_model()
    _check(_lib().ipa_model_init(ctypes.byref(m), kind, t_lo, t_hi), "ipa_model_init")
    return m


def model_1d(t_lo: float = 0.3, t_hi: float = 15.0) -> C.ipa_model:
    return ipa_model_init(C.IPA_MODEL_TIME1D, t_lo, t_hi)


def model_4d(t_lo: float = 0.0, t_hi: float = 15.0) -> C.ipa_model:
    return ipa_model_init(C.IPA_MODEL_ANGTIME4D, t_lo, t_hi)


def model_tagged(t_lo: float = 0.0, t_hi: float = 15.0) -> C.ipa_model:
    return ipa_model_init(C.IPA_MODEL_TAGGED1D, t_lo, t_hi)


def model_phis(t_lo: float = 0.0, t_hi: float = 15.0) -> C.ipa_model:
    """The time-dependent angular model with flavour tagging (16 parameters)."""
    return ipa_model_init(C.IPA_MODEL_PHIS, t_lo, t_hi)


def ipa_events(ev: dict) -> C.ipa_events:
    """dict of CUDA float64 columns (t[, ck, cl, phi][, q][, w][, fk]) -> ipa_events.

    fk, if present, is the (10, stride) tensor written by ipa_angular_basis."""
    t = ev["t"]
    e = C.ipa_events()
    e.n = int(t.numel())
    e.t = _ptr(t, name="t")
    for k in ("ck", "cl", "phi", "w", "q"):
        v = ev.get(k)
        setattr(e, k, _ptr(v, name=k) if v is not None else None)
    fk = ev.get("fk")
    if fk is not None:
        if fk.dim() != 2 or fk.shape[0] != 10:
            raise IpaError("fk must be the (10, stride) angular basis")
        e.fk = _ptr(fk, name="fk")
        e.fk_stride = int(fk.shape[1])
    return e


def ipa_angular_basis(model: C.ipa_model, ev: dict, stream=None) -> torch.Tensor:
    """The 10 angular functions of every event, as a (10, stride) tensor (stride = n rounded
    up to even); put it in the event dict as "fk" to let later calls read it."""
    n = int(ev["t"].numel())
    fk = torch.empty(10, n + (n & 1), dtype=torch.float64, device=ev["t"].device)
    e = ipa_events({k: v for k, v in ev.items() if k != "fk"})
    _check(_lib().ipa_angular_basis(ctypes.byref(model), ctypes.byref(e), _ptr(fk, name="fk"),
                                    int(fk.shape[1]), _stream(stream)), "ipa_angular_basis")
    return fk


def ipa_nll(model: C.ipa_model, ev: dict, theta: torch.Tensor, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    out = torch.empty(1, dtype=torch.float64, device=theta.device) if out is None else out
    _need(theta, model.n_par, "theta")
    _need(out, 1, "out")
    e = ipa_events(ev)
    _check(_lib().ipa_nll(ctypes.byref(model), ctypes.byref(e), _ptr(theta, name="theta"),
                          _ptr(out, name="out"), _stream(stream)), "ipa_nll")
    return out


def ipa_nll_grad(model: C.ipa_model, ev: dict, theta: torch.Tensor, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    out = torch.empty(1 + model.n_par, dtype=torch.float64, device=theta.device) if out is None else out
    _need(theta, model.n_par, "theta")
    _need(out, 1 + model.n_par, "out")
    e = ipa_events(ev)
    _check(_lib().ipa_nll_grad(ctypes.byref(model), ctypes.byref(e), _ptr(theta, name="theta"),
                               _ptr(out, name="out"), _stream(stream)), "ipa_nll_grad")
    return out


def ipa_nll_grad_host(model: C.ipa_model, ev_host: dict, theta: torch.Tensor, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """ipa_nll_grad for events in host memory (CPU float64 tensors, page-locked for
    overlap): chunked copies overlapped with the event pass; the host tensors
    must stay unchanged until the work on the stream completes."""
    out = torch.empty(1 + model.n_par, dtype=torch.float64, device=theta.device) if out is None else out
    _need(theta, model.n_par, "theta")
    _need(out, 1 + model.n_par, "out")
    e = C.ipa_events()
    n = None
    for k in ("t", "ck", "cl", "phi", "w", "q"):
        v = ev_host.get(k)
        if v is None:
            continue
        if not isinstance(v, torch.Tensor) or v.is_cuda or v.dtype != torch.float64 or not v.is_contiguous():
            raise IpaError(f"{k} must be a contiguous float64 CPU tensor")
        n = v.numel() if n is None else n
        if v.numel() != n:
            raise IpaError("host columns of different lengths")
        setattr(e, k, v.data_ptr())
    e.n = 0 if n is None else n
    _check(_lib().ipa_nll_grad_host(ctypes.byref(model), ctypes.byref(e), _ptr(theta, name="theta"),
                                    _ptr(out, name="out"), _stream(stream)), "ipa_nll_grad_host")
    return out


def ipa_nll_grad_noalloc(model: C.ipa_model, ev: dict, theta: torch.Tensor, out: torch.Tensor,
                         stream=None) -> torch.Tensor:
    """ipa_nll_grad with the library's fixed scratch array: allocates nothing on the
    device (the caller passes `out`); at most IPA_NOALLOC_MAX_EVENTS events."""
    _need(theta, model.n_par, "theta")
    _need(out, 1 + model.n_par, "out")
    e = ipa_events(ev)
    _check(_lib().ipa_nll_grad_noalloc(ctypes.byref(model), ctypes.byref(e), _ptr(theta, name="theta"),
                                       _ptr(out, name="out"), _stream(stream)), "ipa_nll_grad_noalloc")
    return out


def ipa_shard_width(model: C.ipa_model) -> int:
    """Doubles per group partial of the event-sharded likelihood."""
    w = ctypes.c_int32(0)
    _check(_lib().ipa_shard_width(ctypes.byref(model), ctypes.byref(w)), "ipa_shard_width")
    return int(w.value)


def shard_groups(n: int) -> int:
    """Group partials of a shard of n events: ceil(n / IPA_SHARD_EVENTS)."""
    return (n + C.IPA_SHARD_EVENTS - 1) // C.IPA_SHARD_EVENTS


def ipa_nll_grad_shard(model: C.ipa_model, ev: dict, theta: torch.Tensor, out: torch.Tensor | None = None,
                       groups: torch.Tensor | None = None, stream=None):
    """This rank's NLL + gradient and its group partials (shard_groups(n) x width)."""
    n = int(ev["t"].numel())
    out = torch.empty(1 + model.n_par, dtype=torch.float64, device=theta.device) if out is None else out
    if groups is None:
        groups = torch.empty(shard_groups(n), ipa_shard_width(model), dtype=torch.float64, device=theta.device)
    _need(theta, model.n_par, "theta")
    _need(out, 1 + model.n_par, "out")
    _need(groups, shard_groups(n) * ipa_shard_width(model), "groups")
    e = ipa_events(ev)
    _check(_lib().ipa_nll_grad_shard(ctypes.byref(model), ctypes.byref(e), _ptr(theta, name="theta"),
                                     _ptr(out, name="out"), _ptr(groups, name="groups") if groups.numel() else None,
                                     _stream(stream)), "ipa_nll_grad_shard")
    return out, groups


def ipa_nll_grad_combine(model: C.ipa_model, theta: torch.Tensor, groups: torch.Tensor, cached: bool = False,
                         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """NLL + gradient from gathered group partials (rows in event order)."""
    out = torch.empty(1 + model.n_par, dtype=torch.float64, device=theta.device) if out is None else out
    _need(theta, model.n_par, "theta")
    _need(out, 1 + model.n_par, "out")
    width = ipa_shard_width(model)
    n_groups = int(groups.numel()) // width
    _check(_lib().ipa_nll_grad_combine(ctypes.byref(model), _ptr(theta, name="theta"),
                                       _ptr(groups, name="groups") if n_groups else None, n_groups, int(cached),
                                       _ptr(out, name="out"), _stream(stream)), "ipa_nll_grad_combine")
    return out


def ipa_nll_grad_segmented(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, theta: torch.Tensor,
                           out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n_seg = int(seg_off.numel()) - 1
    if out is None:
        out = torch.empty(n_seg, 1 + model.n_par, dtype=torch.float64, device=theta.device)
    _need(theta, n_seg * model.n_par, "theta")
    _need(out, n_seg * (1 + model.n_par), "out")
    e = ipa_events(ev)
    _check(_lib().ipa_nll_grad_segmented(ctypes.byref(model), ctypes.byref(e),
                                         _ptr(seg_off, torch.int64, "seg_off"), n_seg,
                                         _ptr(theta, name="theta"), _ptr(out, name="out"),
                                         _stream(stream)), "ipa_nll_grad_segmented")
    return out


def ipa_toygen(model: C.ipa_model, theta: torch.Tensor, seed: int, n_sig: torch.Tensor,
               n_bkg: torch.Tensor, offsets: torch.Tensor, out: dict, stream=None) -> dict:
    """Fill the columns of `out` (dict of CUDA float64 tensors of equal length)."""
    b = C.ipa_event_buffers()
    b.capacity = int(out["t"].numel())
    for k in ("t", "ck", "cl", "phi", "q"):
        v = out.get(k)
        setattr(b, k, _ptr(v, name=k) if v is not None else None)
    _check(_lib().ipa_toygen(ctypes.byref(model), _ptr(theta, name="theta"), ctypes.c_uint64(seed),
                             int(n_sig.numel()), _ptr(n_sig, torch.int64, "n_sig"),
                             _ptr(n_bkg, torch.int64, "n_bkg"), _ptr(offsets, torch.int64, "offsets"),
                             ctypes.byref(b), _stream(stream)), "ipa_toygen")
    return out


@dataclass
class Param:
    """Parameter / Free (App. B): start value, limits, step and the fixed flag."""
    value: float
    lo: float = -1e300
    hi: float = 1e300
    step: float = 0.0
    fixed: bool = False


def _spec(params: list[Param]):
    arr = (C.ipa_param * len(params))()
    for i, p in enumerate(params):
        arr[i].value, arr[i].lo, arr[i].hi = p.value, p.lo, p.hi
        arr[i].step = p.step if p.step > 0 else (
            (p.hi - p.lo) / 10 if p.hi < 1e299 and p.lo > -1e299 else 0.0)
        arr[i].fixed = 1 if p.fixed else 0
    return arr


def ipa_fit_state_bytes(n_fits: int, n_par: int) -> int:
    return int(_lib().ipa_fit_state_bytes(n_fits, n_par))


def fit_state_new(n_fits: int, n_par: int, device) -> torch.Tensor:
    """A zeroed uint8 CUDA buffer for the state of n_fits stepwise fits (the
    caching allocator's blocks are 512-byte aligned)."""
    return torch.zeros(ipa_fit_state_bytes(n_fits, n_par), dtype=torch.uint8, device=device)


def fit_state_points(state: torch.Tensor, n_fits: int, n_par: int) -> torch.Tensor:
    """View of the points the fits want evaluated next (the state's first rows)."""
    return state[:8 * n_fits * n_par].view(torch.float64).view(n_fits, n_par)


def ipa_fit_begin(model: C.ipa_model, params: list[Param], theta0: torch.Tensor, state: torch.Tensor,
                  max_iter: int = 100, tol: float = 1e-9, stream=None):
    n_fits = int(theta0.numel()) // model.n_par
    _need(state, ipa_fit_state_bytes(n_fits, model.n_par), "state")
    _check(_lib().ipa_fit_begin(ctypes.byref(model), _spec(params), n_fits, _ptr(theta0, name="theta0"),
                                max_iter, tol, _ptr(state, torch.uint8, "state"), _stream(stream)), "ipa_fit_begin")


def ipa_fit_advance(model: C.ipa_model, n_fits: int, results: torch.Tensor, state: torch.Tensor,
                    n_active: torch.Tensor, stream=None):
    _need(results, n_fits * (1 + model.n_par), "results")
    _check(_lib().ipa_fit_advance(ctypes.byref(model), n_fits, _ptr(results, name="results"),
                                  _ptr(state, torch.uint8, "state"), _ptr(n_active, torch.int32, "n_active"),
                                  _stream(stream)), "ipa_fit_advance")


def ipa_fit_end(model: C.ipa_model, n_fits: int, state: torch.Tensor, stream=None) -> dict:
    dev = state.device
    out = {"theta": torch.empty(n_fits, model.n_par, dtype=torch.float64, device=dev),
           "err": torch.empty(n_fits, model.n_par, dtype=torch.float64, device=dev),
           "nll": torch.empty(n_fits, dtype=torch.float64, device=dev),
           "status": torch.empty(n_fits, dtype=torch.int32, device=dev),
           "iters": torch.empty(n_fits, dtype=torch.int32, device=dev),
           "passes": torch.empty(n_fits, dtype=torch.int32, device=dev)}
    _check(_lib().ipa_fit_end(ctypes.byref(model), n_fits, _ptr(state, torch.uint8, "state"),
                              _ptr(out["theta"], name="theta"), _ptr(out["err"], name="err"),
                              _ptr(out["nll"], name="nll"), _ptr(out["status"], torch.int32, "status"),
                              _ptr(out["iters"], torch.int32, "iters"), _ptr(out["passes"], torch.int32, "passes"),
                              _stream(stream)), "ipa_fit_end")
    return out


def ipa_fit_batch(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, params: list[Param],
                  theta: torch.Tensor, max_iter: int = 100, tol: float = 1e-9, stream=None) -> dict:
    """Fit every segment; theta (n_fits x n_par) holds the start values and receives the result."""
    n_fits = int(seg_off.numel()) - 1
    dev = theta.device
    err = torch.zeros(n_fits, model.n_par, dtype=torch.float64, device=dev)
    nll = torch.zeros(n_fits, dtype=torch.float64, device=dev)
    status = torch.zeros(n_fits, dtype=torch.int32, device=dev)
    iters = torch.zeros(n_fits, dtype=torch.int32, device=dev)
    passes = torch.zeros(n_fits, dtype=torch.int32, device=dev)
    e = ipa_events(ev)
    spec = _spec(params)
    _check(_lib().ipa_fit_batch(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"),
                                n_fits, spec, _ptr(theta, name="theta"), _ptr(err, name="err"),
                                _ptr(nll, name="nll"), _ptr(status, torch.int32, "status"),
                                _ptr(iters, torch.int32, "iters"), _ptr(passes, torch.int32, "passes"),
                                max_iter, tol, _stream(stream)),
           "ipa_fit_batch")
    return {"theta": theta, "err": err, "nll": nll, "status": status, "iters": iters, "passes": passes}


class Joint:
    """A simultaneous fit's category map (Sec. 4 Example 2; App. B, Cat and
    ParamBox): jmap[c][p] is the joint parameter that model parameter p of
    category c takes, or -1 for the constant value[c][p]."""

    def __init__(self, jmap, value=None, n_joint: int | None = None):
        self.map = np.ascontiguousarray(np.asarray(jmap, dtype=np.int32))
        if self.map.ndim != 2:
            raise ValueError("the joint map is n_cat x n_par")
        self.value = None if value is None else np.ascontiguousarray(np.asarray(value, dtype=np.float64))
        if self.value is not None and self.value.shape != self.map.shape:
            raise ValueError("the joint values have the map's shape")
        self.n_cat = self.map.shape[0]
        self.n_joint = int(self.map.max()) + 1 if n_joint is None else int(n_joint)

    def c_struct(self) -> C.ipa_joint:
        j = C.ipa_joint()
        j.n_cat, j.n_joint = self.n_cat, self.n_joint
        j.map = self.map.ctypes.data
        j.value = None if self.value is None else self.value.ctypes.data
        return j


def ipa_nll_grad_joint(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, joint: Joint, theta: torch.Tensor,
                       stream=None) -> torch.Tensor:
    """Joint NLL and gradient of n_fits simultaneous fits (theta: n_fits x n_joint;
    segment i * n_cat + c is category c of fit i): an (n_fits, 1 + n_joint) tensor."""
    n_seg = int(seg_off.numel()) - 1
    if n_seg % joint.n_cat:
        raise ValueError("the segments are not a whole number of fits")
    n_fits = n_seg // joint.n_cat
    _need(theta, n_fits * joint.n_joint, "theta")
    if joint.map.shape[1] != model.n_par:
        raise ValueError("the joint map has a column per model parameter")
    out = torch.empty(n_fits, 1 + joint.n_joint, dtype=torch.float64, device=theta.device)
    e, j = ipa_events(ev), joint.c_struct()
    _check(_lib().ipa_nll_grad_joint(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"),
                                     n_fits, ctypes.byref(j), _ptr(theta, name="theta"), _ptr(out, name="out"),
                                     _stream(stream)),
           "ipa_nll_grad_joint")
    return out


def ipa_fit_joint(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, joint: Joint, params: list[Param],
                  theta: torch.Tensor, max_iter: int = 100, tol: float = 1e-9, stream=None) -> dict:
    """Fit n_fits simultaneous fits; params: the n_joint joint parameters; theta
    (n_fits x n_joint) holds the start values and receives the result."""
    n_seg = int(seg_off.numel()) - 1
    if n_seg % joint.n_cat or len(params) != joint.n_joint:
        raise ValueError("segments or parameters do not match the joint map")
    n_fits = n_seg // joint.n_cat
    _need(theta, n_fits * joint.n_joint, "theta")
    if joint.map.shape[1] != model.n_par:
        raise ValueError("the joint map has a column per model parameter")
    dev = theta.device
    err = torch.zeros(n_fits, joint.n_joint, dtype=torch.float64, device=dev)
    nll = torch.zeros(n_fits, dtype=torch.float64, device=dev)
    status = torch.zeros(n_fits, dtype=torch.int32, device=dev)
    iters = torch.zeros(n_fits, dtype=torch.int32, device=dev)
    passes = torch.zeros(n_fits, dtype=torch.int32, device=dev)
    e, j, spec = ipa_events(ev), joint.c_struct(), _spec(params)
    _check(_lib().ipa_fit_joint(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"),
                                n_fits, ctypes.byref(j), spec, _ptr(theta, name="theta"), _ptr(err, name="err"),
                                _ptr(nll, name="nll"), _ptr(status, torch.int32, "status"),
                                _ptr(iters, torch.int32, "iters"), _ptr(passes, torch.int32, "passes"),
                                max_iter, tol, _stream(stream)),
           "ipa_fit_joint")
    return {"theta": theta, "err": err, "nll": nll, "status": status, "iters": iters, "passes": passes}


def ipa_hesse(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, params: list[Param],
              theta: torch.Tensor, stream=None) -> dict:
    """Covariance, correlation matrix, errors and status of each fit at theta (n_fits x n_par)."""
    n_fits = int(seg_off.numel()) - 1
    P = model.n_par
    dev = theta.device
    cov = torch.empty(n_fits, P, P, dtype=torch.float64, device=dev)
    corr = torch.empty(n_fits, P, P, dtype=torch.float64, device=dev)
    err = torch.empty(n_fits, P, dtype=torch.float64, device=dev)
    status = torch.empty(n_fits, dtype=torch.int32, device=dev)
    e = ipa_events(ev)
    _check(_lib().ipa_hesse(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"), n_fits,
                            _spec(params), _ptr(theta, name="theta"), _ptr(cov, name="cov"),
                            _ptr(corr, name="corr"), _ptr(err, name="err"), _ptr(status, torch.int32, "status"),
                            _stream(stream)), "ipa_hesse")
    return {"cov": cov, "corr": corr, "err": err, "status": status}


def ipa_hesse_joint(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, joint: Joint, params: list[Param],
                    theta: torch.Tensor, stream=None) -> dict:
    """Covariance, correlation matrix, errors and status of each simultaneous
    fit at theta (n_fits x n_joint)."""
    n_seg = int(seg_off.numel()) - 1
    if n_seg % joint.n_cat or len(params) != joint.n_joint or joint.map.shape[1] != model.n_par:
        raise ValueError("segments, parameters or map do not match the joint map")
    n_fits = n_seg // joint.n_cat
    P = joint.n_joint
    _need(theta, n_fits * P, "theta")
    dev = theta.device
    cov = torch.empty(n_fits, P, P, dtype=torch.float64, device=dev)
    corr = torch.empty(n_fits, P, P, dtype=torch.float64, device=dev)
    err = torch.empty(n_fits, P, dtype=torch.float64, device=dev)
    status = torch.empty(n_fits, dtype=torch.int32, device=dev)
    e, j = ipa_events(ev), joint.c_struct()
    _check(_lib().ipa_hesse_joint(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"),
                                  n_fits, ctypes.byref(j), _spec(params), _ptr(theta, name="theta"),
                                  _ptr(cov, name="cov"), _ptr(corr, name="corr"), _ptr(err, name="err"),
                                  _ptr(status, torch.int32, "status"), _stream(stream)), "ipa_hesse_joint")
    return {"cov": cov, "corr": corr, "err": err, "status": status}


def ipa_minos(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, params: list[Param], theta_min: torch.Tensor,
              nll_min: torch.Tensor, cov: torch.Tensor, scan: list[int], up: float = 0.5, tol: float = 1e-7,
              max_rounds: int = 12, max_iter: int = 200, fit_tol: float = 1e-9, stream=None) -> dict:
    """MINOS intervals (lower and upper signed errors, statuses) of the parameters in `scan`."""
    n_fits = int(seg_off.numel()) - 1
    P = model.n_par
    dev = theta_min.device
    lo = torch.empty(n_fits, P, dtype=torch.float64, device=dev)
    hi = torch.empty(n_fits, P, dtype=torch.float64, device=dev)
    status = torch.empty(n_fits, P, 2, dtype=torch.int32, device=dev)
    flags = (ctypes.c_int32 * P)(*[1 if p in scan else 0 for p in range(P)])
    e = ipa_events(ev)
    _check(_lib().ipa_minos(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"), n_fits,
                            _spec(params), _ptr(theta_min, name="theta_min"), _ptr(nll_min, name="nll_min"),
                            _ptr(cov, name="cov"), flags, up, tol, max_rounds, max_iter, fit_tol,
                            _ptr(lo, name="lo"), _ptr(hi, name="hi"), _ptr(status, torch.int32, "status"),
                            _stream(stream)), "ipa_minos")
    return {"lo": lo, "hi": hi, "status": status}


def ipa_minos_joint(model: C.ipa_model, ev: dict, seg_off: torch.Tensor, joint: Joint, params: list[Param],
                    theta_min: torch.Tensor, nll_min: torch.Tensor, cov: torch.Tensor, scan: list[int],
                    up: float = 0.5, tol: float = 1e-7, max_rounds: int = 12, max_iter: int = 200,
                    fit_tol: float = 1e-9, stream=None) -> dict:
    """MINOS intervals of the joint parameters in `scan` of simultaneous fits."""
    n_seg = int(seg_off.numel()) - 1
    if n_seg % joint.n_cat or len(params) != joint.n_joint or joint.map.shape[1] != model.n_par:
        raise ValueError("segments, parameters or map do not match the joint map")
    n_fits = n_seg // joint.n_cat
    P = joint.n_joint
    _need(theta_min, n_fits * P, "theta_min")
    _need(nll_min, n_fits, "nll_min")
    _need(cov, n_fits * P * P, "cov")
    dev = theta_min.device
    lo = torch.empty(n_fits, P, dtype=torch.float64, device=dev)
    hi = torch.empty(n_fits, P, dtype=torch.float64, device=dev)
    status = torch.empty(n_fits, P, 2, dtype=torch.int32, device=dev)
    flags = (ctypes.c_int32 * P)(*[1 if p in scan else 0 for p in range(P)])
    e, j = ipa_events(ev), joint.c_struct()
    _check(_lib().ipa_minos_joint(ctypes.byref(model), ctypes.byref(e), _ptr(seg_off, torch.int64, "seg_off"),
                                  n_fits, ctypes.byref(j), _spec(params), _ptr(theta_min, name="theta_min"),
                                  _ptr(nll_min, name="nll_min"), _ptr(cov, name="cov"), flags, up, tol, max_rounds,
                                  max_iter, fit_tol, _ptr(lo, name="lo"), _ptr(hi, name="hi"),
                                  _ptr(status, torch.int32, "status"), _stream(stream)), "ipa_minos_joint")
    return {"lo": lo, "hi": hi, "status": status}


def ipa_binned_generate(lam: torch.Tensor, seed: int, n_toys: int, toy0: int = 0, hypothesis: int = 0,
                        stream=None) -> torch.Tensor:
    """(n_toys, n_bins) int32 Poisson counts of the bin means lam (generateBinned)."""
    n_bins = int(lam.numel())
    out = torch.empty(n_toys, n_bins, dtype=torch.int32, device=lam.device)
    _check(_lib().ipa_binned_generate(_ptr(lam, name="lambda"), n_bins, ctypes.c_uint64(seed), hypothesis, toy0,
                                      n_toys, _ptr(out, torch.int32, "counts"), _stream(stream)),
           "ipa_binned_generate")
    return out


def ipa_binned_smear(hist: torch.Tensor, bin_width: float, sigma: float, stream=None) -> torch.Tensor:
    """The histogram convolved with a Gaussian of width sigma (same binning)."""
    out = torch.empty_like(hist)
    _check(_lib().ipa_binned_smear(_ptr(hist, name="hist"), int(hist.numel()), bin_width, sigma,
                                   _ptr(out, name="out"), _stream(stream)), "ipa_binned_smear")
    return out


def ipa_cls(s: torch.Tensor, b: torch.Tensor, data: torch.Tensor, n_toys: int, seed: int, with_x: bool = False,
            stream=None) -> dict:
    """CL_b, CL_s+b, CL_s of the observed counts `data` (int32) for signal s over background b."""
    n_bins = int(s.numel())
    cl = torch.empty(3, dtype=torch.float64, device=s.device)
    counts = torch.empty(2, dtype=torch.int64, device=s.device)
    x = torch.empty(2 * n_toys + 1, dtype=torch.float64, device=s.device) if with_x else None
    _check(_lib().ipa_cls(_ptr(s, name="s"), _ptr(b, name="b"), n_bins, _ptr(data, torch.int32, "data"), n_toys,
                          ctypes.c_uint64(seed), _ptr(cl, name="cl"), _ptr(counts, torch.int64, "counts"),
                          _ptr(x, name="x") if x is not None else None, _stream(stream)), "ipa_cls")
    out = {"cl_b": cl[0], "cl_sb": cl[1], "cl_s": cl[2], "counts": counts}
    if x is not None:
        out["x_b"], out["x_sb"], out["x_obs"] = x[:n_toys], x[n_toys:2 * n_toys], x[2 * n_toys]
    return out


def _host_or_dev_ptr(x, name):
    """Pointer of a C-contiguous float64 numpy array (host) or CUDA tensor (device)."""
    import numpy as np
    if isinstance(x, torch.Tensor):
        return _ptr(x, name=name), int(x.numel())
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise IpaError(f"{name} must be a contiguous float64 numpy array or CUDA tensor")
    return x.ctypes.data, int(x.size)


def ipa_server_create(model: C.ipa_model, hbm_budget_bytes: int, max_slots: int = 256,
                      max_iter: int = 200, tol: float = 1e-8) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib().ipa_server_create(ctypes.byref(model), hbm_budget_bytes, max_slots, max_iter, tol,
                                    ctypes.byref(h)), "ipa_server_create")
    return h


def ipa_serve_submit(server, ev: dict, params: list[Param]) -> int:
    """Submit one fit; ev holds host numpy arrays or CUDA tensors (copied before return)."""
    e = C.ipa_events()
    keep = []
    for k in ("t", "ck", "cl", "phi", "w", "q"):
        v = ev.get(k)
        if v is None:
            setattr(e, k, None)
            continue
        ptr, n = _host_or_dev_ptr(v, k)
        keep.append(v)
        setattr(e, k, ptr)
        if k == "t":
            e.n = n
    ticket = ctypes.c_uint64()
    _check(_lib().ipa_serve_submit(server, ctypes.byref(e), _spec(params), ctypes.byref(ticket)),
           "ipa_serve_submit")
    return ticket.value


def ipa_serve_poll(server, ticket: int, n_par: int):
    """None while the fit is pending; else dict(theta, err, nll, status)."""
    import numpy as np
    th = (ctypes.c_double * n_par)()
    er = (ctypes.c_double * n_par)()
    nll = ctypes.c_double()
    st = ctypes.c_int32()
    r = _lib().ipa_serve_poll(server, ctypes.c_uint64(ticket), th, er, ctypes.byref(nll), ctypes.byref(st))
    if r == C.IPA_PENDING:
        return None
    _check(r, "ipa_serve_poll")
    return {"theta": np.array(th[:]), "err": np.array(er[:]), "nll": nll.value, "status": st.value}


def ipa_server_destroy(server):
    _check(_lib().ipa_server_destroy(server), "ipa_server_destroy")


def ipa_reserve(max_events: int, max_segments: int = 1):
    _check(_lib().ipa_reserve(max_events, max_segments), "ipa_reserve")


def ipa_fault_inject(mask: int) -> int:
    """Set the host-side fault-injection mask (IPA_FAULT_*); returns the previous one."""
    return int(_lib().ipa_fault_inject(mask))


def ipa_scratch_bytes() -> int:
    """Device bytes held by the library's per-device scratch on the current device."""
    v = ctypes.c_uint64(0)
    _check(_lib().ipa_scratch_bytes(ctypes.byref(v)), "ipa_scratch_bytes")
    return int(v.value)


def _cfg_dict(c: C.ipa_launch_config) -> dict:
    return {"warps_per_block": c.warps_per_block, "warps_per_sm": c.warps_per_sm,
            "tiles_per_take": c.tiles_per_take, "ms": float(c.ms)}


def ipa_autotune(model: C.ipa_model, ev: dict, theta: torch.Tensor, grad: bool = True,
                 seg_off: torch.Tensor | None = None, stream=None) -> dict:
    """Time every launch geometry of the likelihood kernel on these events and keep
    the fastest for their size class (results never depend on the geometry)."""
    n_seg = 1 if seg_off is None else int(seg_off.numel()) - 1
    picked = C.ipa_launch_config()
    e = ipa_events(ev)
    _check(_lib().ipa_autotune(ctypes.byref(model), ctypes.byref(e),
                               None if seg_off is None else _ptr(seg_off, torch.int64, "seg_off"), n_seg,
                               _ptr(theta, name="theta"), int(bool(grad)), ctypes.byref(picked),
                               _stream(stream)), "ipa_autotune")
    return _cfg_dict(picked)


def ipa_launch_config_get(model: C.ipa_model, n_events: int, n_seg: int = 1, grad: bool = True,
                          cached: bool = False) -> dict:
    c = C.ipa_launch_config()
    _check(_lib().ipa_launch_config_get(ctypes.byref(model), n_events, n_seg, int(bool(grad)), int(bool(cached)),
                                        ctypes.byref(c)), "ipa_launch_config_get")
    return _cfg_dict(c)


def ipa_launch_config_set(model: C.ipa_model, n_events: int, cfg: dict, n_seg: int = 1, grad: bool = True,
                          cached: bool = False):
    c = C.ipa_launch_config(int(cfg["warps_per_block"]), int(cfg["warps_per_sm"]), int(cfg["tiles_per_take"]),
                            0.0)
    _check(_lib().ipa_launch_config_set(ctypes.byref(model), n_events, n_seg, int(bool(grad)), int(bool(cached)),
                                        ctypes.byref(c)), "ipa_launch_config_set")


def ipa_calibrate_fp64(stream=None) -> dict:
    """DFMA rate and FP64 math-function costs of the current GPU (see the header)."""
    r = (ctypes.c_double * 15)()
    _check(_lib().ipa_calibrate_fp64(r, _stream(stream)), "ipa_calibrate_fp64")
    names = ["dfma_per_clk_per_sm", "dfma_per_s", "exp", "erfc", "log", "sincos", "sqrt", "rcp", "sm_mhz",
             "exp_fast", "log_fast", "sincos_fast", "erfcx_poly", "exp_int", "sincos_int"]
    return dict(zip(names, list(r)))


def ipa_math_eval(fn: int, x: torch.Tensor, stream=None) -> torch.Tensor:
    """The library's own FP64 function `fn` (C.IPA_MATH_*) elementwise on a CUDA tensor."""
    y = torch.empty_like(x)
    _check(_lib().ipa_math_eval(int(fn), _ptr(x, name="x"), _ptr(y, name="y"), x.numel(), _stream(stream)),
           "ipa_math_eval")
    return y


def ipa_faddeeva(z: torch.Tensor, stream=None) -> torch.Tensor:
    """w(z) = exp(-z^2) erfc(-i z) elementwise, as the tagged model's kernels evaluate it;
    z is a complex128 CUDA tensor."""
    if not (isinstance(z, torch.Tensor) and z.is_cuda and z.dtype == torch.complex128):
        raise IpaError("z must be a complex128 CUDA tensor")
    zr = torch.view_as_real(z.contiguous()).contiguous()
    wr = torch.empty_like(zr)
    _check(_lib().ipa_faddeeva(zr.data_ptr(), wr.data_ptr(), z.numel(), _stream(stream)), "ipa_faddeeva")
    return torch.view_as_complex(wr)


def ipa_version() -> str:
    return _lib().ipa_version().decode()
