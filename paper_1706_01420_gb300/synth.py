"""Seeded synthetic inputs shared by the tests, the benchmark and the examples.

This module draws random numbers only.  It evaluates no probability density,
normalisation, likelihood or amplitude: every event column comes from numpy's
samplers (exponential, normal, uniform, Poisson, binomial), so it can serve
both the CUDA path and the CPU oracle without carrying either side's
arithmetic.  The recipes stand in for the EvtGen / LHCb samples of the paper
(Examples 1, 2 and 5), which are not available.

Recipes (all FP64, structure-of-arrays, one numpy Generator per call):

* decay time:  each event is background with probability ``f_b`` (a flat
  time) and signal otherwise: ``s + e`` with ``s ~ Exp(rate Gamma)`` and
  ``e ~ Normal(mu, sigma)``, redrawn until it falls inside ``[t_lo, t_hi]``,
  so the class fractions are those of the truncated mixture.
* angles: ``cos(theta_K)``, ``cos(theta_mu)`` uniform on [-1, 1] and ``phi``
  uniform on [-pi, pi] (the flat-acceptance ranges of the helicity angles).
  Events distributed like the full angular PDF come from the toy generator
  instead (``ipa_toygen`` on the GPU, the oracle's generator on the CPU).
* flavour tags (tagged model): ``q = +1`` or ``-1`` with probability 1/2 each,
  independent of the time (a tag-blind sample; tagged samples distributed like
  the model come from the generators, as for the angles).
* weights: ``Normal(1, 0.2)``, the per-event weights of the serving workload.
* toy sizes: ``N_k ~ Poisson(mean)`` per toy, then ``n_bkg ~ Binomial(N_k,
  f_b)``; the split is drawn on the host, as Example 5 of the paper advises
  for the event counts, and passed to both generators as an input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TRUTH_1D = {"Gamma": 0.66, "sigma": 0.045, "mu": 0.0, "f_b": 0.1}
TRUTH_4D = {
    "Gamma": 0.66, "sigma": 0.045, "mu": 0.0, "f_b": 0.1,
    "A0sq": 0.52, "Apesq": 0.25, "delta_pa": 3.2, "delta_pe": 3.1,
    "F_S": 0.04, "delta_S": 0.3,
}


def _times(rng: np.random.Generator, n: int, t_lo: float, t_hi: float,
           Gamma: float, sigma: float, mu: float, f_b: float) -> np.ndarray:
    """Class first (background with probability f_b), then a time of that class
    inside [t_lo, t_hi]; signal times are redrawn until they fall in the range,
    so the class fractions hold after the truncation."""
    is_bkg = rng.random(n) < f_b
    n_bkg = int(is_bkg.sum())
    out = np.empty(n, dtype=np.float64)
    out[is_bkg] = rng.uniform(t_lo, t_hi, n_bkg)
    sig = np.empty(n - n_bkg, dtype=np.float64)
    filled = 0
    while filled < sig.size:
        m = max(1024, int(1.5 * (sig.size - filled)))
        t = rng.exponential(1.0 / Gamma, m) + rng.normal(mu, sigma, m)
        t = t[(t >= t_lo) & (t <= t_hi)]
        take = min(t.size, sig.size - filled)
        sig[filled:filled + take] = t[:take]
        filled += take
    out[~is_bkg] = sig
    return out


def events_1d(n: int, seed: int = 0, t_lo: float = 0.3, t_hi: float = 15.0,
              truth: dict | None = None) -> np.ndarray:
    """Decay times for the one-dimensional workload (config: 1e5 events on [0.3, 15] ps)."""
    p = dict(TRUTH_1D if truth is None else truth)
    rng = np.random.default_rng(seed)
    return _times(rng, n, t_lo, t_hi, p["Gamma"], p["sigma"], p["mu"], p["f_b"])


def events_4d(n: int, seed: int = 0, t_lo: float = 0.0, t_hi: float = 15.0,
              truth: dict | None = None, weighted: bool = False) -> dict:
    """SoA columns t, ck, cl, phi (and w) for the angular+time workload."""
    p = dict(TRUTH_4D if truth is None else truth)
    rng = np.random.default_rng(seed)
    t = _times(rng, n, t_lo, t_hi, p["Gamma"], p["sigma"], p["mu"], p["f_b"])
    ck = rng.uniform(-1.0, 1.0, n)
    cl = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(-math.pi, math.pi, n)
    cols = {"t": t, "ck": ck, "cl": cl, "phi": phi}
    if weighted:
        cols["w"] = weights(n, seed + 7919)
    return cols


TRUTH_TAGGED = {"Gamma": 0.66, "sigma": 0.045, "mu": 0.0, "f_b": 0.1,
                "DG": 0.085, "Dm": 17.77, "phi_s": 0.8, "omega": 0.3}


def events_tagged(n: int, seed: int = 0, t_lo: float = 0.0, t_hi: float = 15.0,
                  truth: dict | None = None, weighted: bool = False) -> dict:
    """SoA columns t, q (and w) for the flavour-tagged workload."""
    p = dict(TRUTH_TAGGED if truth is None else truth)
    rng = np.random.default_rng(seed)
    t = _times(rng, n, t_lo, t_hi, p["Gamma"], p["sigma"], p["mu"], p["f_b"])
    q = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    cols = {"t": t, "q": q}
    if weighted:
        cols["w"] = weights(n, seed + 7919)
    return cols


def events_phis(n: int, seed: int = 0, t_lo: float = 0.0, t_hi: float = 15.0, truth: dict | None = None,
                weighted: bool = False) -> dict:
    """SoA columns t, ck, cl, phi, q (and w) for the time-dependent angular model
    with tagging: the 4D recipe plus a tag-blind q."""
    cols = events_4d(n, seed, t_lo=t_lo, t_hi=t_hi, truth=truth, weighted=weighted)
    rng = np.random.default_rng(seed + 104729)
    cols["q"] = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    return cols


def weights(n: int, seed: int = 0, mean: float = 1.0, sd: float = 0.2) -> np.ndarray:
    """Per-event weights ~ Normal(mean, sd)."""
    return np.random.default_rng(seed).normal(mean, sd, n)


def toy_sizes(n_toys: int, mean: float, f_b: float, seed: int = 0):
    """Per-toy signal and background counts: N_k ~ Poisson(mean), n_bkg ~ Binomial(N_k, f_b)."""
    rng = np.random.default_rng(seed)
    n_tot = rng.poisson(mean, n_toys).astype(np.int64)
    n_bkg = rng.binomial(n_tot, f_b).astype(np.int64)
    return n_tot - n_bkg, n_bkg


@dataclass
class FitRequest:
    arrival_s: float
    n_events: int
    seed: int


def request_stream(n_requests: int, rate_hz: float, n_lo: float = 1e3, n_hi: float = 1e7,
                   seed: int = 0) -> list[FitRequest]:
    """Poisson arrivals at ``rate_hz`` with event counts log-uniform on [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    arrivals = np.cumsum(gaps)
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_requests)).astype(np.int64)
    return [FitRequest(float(a), int(s), int(seed * 1_000_003 + i))
            for i, (a, s) in enumerate(zip(arrivals, sizes))]
