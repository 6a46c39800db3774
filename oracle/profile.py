"""Plain FP64 CPU oracle of the error analysis after a fit: the HESSE
covariance and the MINOS (profile-likelihood) intervals.  Test infrastructure
only, like the rest of ``oracle/``: only tests, the smoke check and the
bench's CPU legs use it.

The method (arXiv:1706.01420):

* Sec. 3 and Sec. 4 (Examples 1 and 2): after MIGRAD, HESSE gives the
  parameter errors and the correlation matrix (Figs. 2 and 4), with the FCN
  = -log L, i.e. errors at Delta(-log L) = 1/2.
* The MINOS interval of a parameter (the MINUIT procedure the paper's fits
  call through iminuit) is where the profile of -log L, minimised over every
  other free parameter, rises by ``up`` = 1/2 above the minimum on each side.

Definitions used here, each written out plainly:

* hesse: H = second derivatives of the NLL over the free parameters by
  central differences of the analytic gradient (``ipa_oracle.hessian_fd``);
  covariance C = H^-1, errors sqrt(C_ii), correlations C_ij / sqrt(C_ii C_jj).
* profile(x): min over the other free parameters of NLL(theta) with theta_j
  fixed at x (``ipa_oracle.fit``), or NLL at x when j is the only free one.
* minos: on each side the root of profile(x) - NLL_min - up, bracketed by
  stepping out from the minimum in multiples of the HESSE error and found by
  Brent's method (scipy.optimize.brentq).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

from . import ipa_oracle as O


def hesse(model: O.Model, ev: dict, theta, free):
    """(covariance over all parameters (zero rows/columns for fixed ones),
    errors, correlation matrix over the free parameters, H over the free ones)."""
    theta = np.asarray(theta, dtype=np.float64)
    free = list(free)
    H = O.hessian_fd(model, ev, theta, free)
    Cf = np.linalg.inv(H)
    n = model.npar
    C = np.zeros((n, n))
    C[np.ix_(free, free)] = Cf
    err = np.sqrt(np.maximum(np.diag(C), 0.0))
    d = np.sqrt(np.diag(Cf))
    corr = Cf / np.outer(d, d)
    return C, err, corr, H


def profile(model: O.Model, ev: dict, theta_hat, free, j: int, x: float, lo=None, hi=None, tol=1e-10):
    """Profile NLL at theta_j = x and the constrained minimum."""
    return profile_function(lambda th: O.nll_grad(model, ev, th), model.npar, theta_hat, free, j, x, lo, hi, tol)


def profile_function(fn, n, theta_hat, free, j: int, x: float, lo=None, hi=None, tol=1e-10):
    """The same for any fn(theta) -> (NLL, gradient) of n parameters."""
    th = np.asarray(theta_hat, dtype=np.float64).copy()
    th[j] = x
    others = [p for p in free if p != j]
    if not others:
        return fn(th)[0], th
    r = O.fit_function(fn, n, th, others, lo=lo, hi=hi, tol=tol, max_iter=100)
    return r.nll, r.theta


def minos(model: O.Model, ev: dict, theta_hat, nll_hat: float, free, j: int, sigma0: float,
          up: float = 0.5, lo=None, hi=None, tol=1e-10):
    """MINOS errors (x_lo - theta_j, x_hi - theta_j) of parameter j and a
    status per side: "OK", or "LIMIT" when the profile stays below the
    threshold up to the parameter's limit (the error then reaches the limit)."""
    return minos_function(lambda th: O.nll_grad(model, ev, th), model.npar, theta_hat, nll_hat, free, j, sigma0,
                          up, lo, hi, tol)


def minos_function(fn, n, theta_hat, nll_hat: float, free, j: int, sigma0: float, up: float = 0.5, lo=None,
                   hi=None, tol=1e-10):
    """The same for any fn(theta) -> (NLL, gradient) of n parameters."""
    theta_hat = np.asarray(theta_hat, dtype=np.float64)
    lo = np.full(n, -np.inf) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.full(n, np.inf) if hi is None else np.asarray(hi, dtype=np.float64)
    c = float(theta_hat[j])

    def excess(x):
        return profile_function(fn, n, theta_hat, free, j, x, lo, hi, tol)[0] - nll_hat - up

    out, status = [0.0, 0.0], ["OK", "OK"]
    for k, side in enumerate((-1.0, 1.0)):
        limit = lo[j] if side < 0 else hi[j]
        step = sigma0
        x = c + side * step
        while True:
            if (side < 0 and x <= limit) or (side > 0 and x >= limit):
                x = limit
                if excess(x) < 0.0:
                    status[k] = "LIMIT"
                    out[k] = x - c
                    break
            if excess(x) > 0.0:
                root = brentq(excess, min(c, x), max(c, x), xtol=1e-12 * sigma0, rtol=1e-14, maxiter=200)
                out[k] = root - c
                break
            step *= 2.0
            x = c + side * step
    return (out[0], out[1]), tuple(status)
