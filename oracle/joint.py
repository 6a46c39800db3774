"""Plain FP64 CPU oracle of a simultaneous fit over categories (test
infrastructure only, like the rest of ``oracle/``: only tests, the smoke check
and the bench's CPU legs use it).

The method (arXiv:1706.01420, Sec. 4, Example 2 and App. B): one -2 log L
summed over categories (Example 2: six m(KK) bins times the two B flavours)
whose parameters are partly shared (the polarisation fractions, the phases,
Gamma, Delta Gamma, Delta m) and partly per category (the S-wave parameters
of each bin), with per-category constants (C_SP).  Reading:

* category c evaluates the model at theta_c, with
  theta_c[p] = theta_J[map[c][p]] where map[c][p] >= 0 and the constant
  value[c][p] where map[c][p] = -1;
* NLL_J(theta_J) = sum_c NLL(theta_c; events of c);
* the gradient by the chain rule of that linear map:
  dNLL_J / dtheta_J[j] = sum over (c, p) with map[c][p] = j of
  dNLL / dtheta_c[p].

The per-category NLL and gradient are the model oracle's (``ipa_oracle``).
"""
from __future__ import annotations

import math

import numpy as np

from . import ipa_oracle as O


def category_thetas(jmap, value, theta_joint) -> np.ndarray:
    """theta_c for every category: an (n_cat, n_par) array."""
    jmap = np.asarray(jmap, dtype=np.int64)
    theta_joint = np.asarray(theta_joint, dtype=np.float64)
    out = np.zeros(jmap.shape)
    for c in range(jmap.shape[0]):
        for p in range(jmap.shape[1]):
            j = int(jmap[c, p])
            out[c, p] = theta_joint[j] if j >= 0 else float(value[c][p])
    return out


def nll_grad(model: O.Model, cats: list, jmap, value, theta_joint):
    """(NLL_J, dNLL_J/dtheta_J) of one simultaneous fit; cats: the categories' event dicts."""
    jmap = np.asarray(jmap, dtype=np.int64)
    n_joint = len(theta_joint)
    ths = category_thetas(jmap, value, theta_joint)
    fs = []
    parts = [[] for _ in range(n_joint)]
    for c, ev in enumerate(cats):
        f, g = O.nll_grad(model, ev, ths[c])
        fs.append(f)
        for p in range(jmap.shape[1]):
            if jmap[c, p] >= 0:
                parts[int(jmap[c, p])].append(float(g[p]))
    return math.fsum(fs), np.array([math.fsum(v) for v in parts])


def nll(model: O.Model, cats: list, jmap, value, theta_joint) -> float:
    return nll_grad(model, cats, jmap, value, theta_joint)[0]


def fit(model: O.Model, cats: list, jmap, value, theta0, free, lo=None, hi=None, tol=1e-10,
        max_iter=100) -> O.FitResult:
    """Minimise NLL_J over the free joint parameters with the model oracle's
    Newton iteration (``ipa_oracle.fit``) applied to the joint function."""
    return O.fit_function(lambda th: nll_grad(model, cats, jmap, value, th), len(theta0), theta0, free, lo=lo,
                          hi=hi, tol=tol, max_iter=max_iter)


def minos(model: O.Model, cats: list, jmap, value, theta_hat, nll_hat: float, free, j: int, sigma0: float,
          up: float = 0.5, lo=None, hi=None, tol=1e-10):
    """MINOS errors of joint parameter j (``profile.minos_function`` applied to
    the joint NLL)."""
    from . import profile
    return profile.minos_function(lambda th: nll_grad(model, cats, jmap, value, th), len(theta_hat), theta_hat,
                                  nll_hat, free, j, sigma0, up, lo, hi, tol)

