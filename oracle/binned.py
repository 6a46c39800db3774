"""Plain FP64 CPU oracle of the binned workloads: Poisson pseudo-experiments
of a histogram, Gaussian smearing of a histogram, and the CLs confidence
levels from toys.  Test infrastructure only, like the rest of ``oracle/``:
only tests, the smoke check and the bench's CPU legs use it.

The method (arXiv:1706.01420, Example 4 "CLs" and the toolkit utilities it
calls): a binned model HistoPdf = ns S + nb B from a smeared signal shape S
and a background shape B (both normalised to unit sum over the bins), a data
histogram drawn from it (generateBinned), and CL_b, CL_s+b and CL_s from
10 000 toy experiments (CLcalculator), the modified frequentist method of
the LEP Higgs searches (the paper's CLs references).

Readings (the paper prints the calls, not the formulas):

* Poisson counts: bin i of toy k is Poisson(lambda_i) by inversion of the
  CDF with one uniform from the counter-based Philox-4x32-10 of
  ``ipa_oracle`` (counters (i lo32, i hi32, k, 8 + 2^16 h + m // 2), words
  2 (m mod 2) and 2 (m mod 2) + 1, key = seed; h = 0 for the
  background-only and 1 for the signal-plus-background hypothesis of CLs, 0
  for plain generation).  A mean above 400 is split into M = ceil(lambda /
  400) pieces of lambda / M (Poisson counts add), piece m using the uniform
  above.  Inversion of one piece of mean nu with uniform u:
      n = 0, p = exp(-nu), F = p;  while u > F and p > 0 and n < cap:
          n = n + 1, p = (p nu) / n, F = F + p,
  cap = floor(nu + 40 sqrt(nu) + 100) (reached only when the floating-point
  CDF stalls below u <= 1).
* Smearing: out_i = sum_d K_d h_{i-d} over |d| <= R = ceil(8 sigma / Delta),
  bins outside the histogram contributing nothing, with the discrete
  Gaussian K_d = e^{-(d Delta)^2 / (2 sigma^2)} / sum_{|d'| <= R} e^{-(d' Delta)^2 / (2 sigma^2)}.
* Test statistic: X = sum_i n_i ln(1 + s_i / b_i) (the data-dependent part
  of -2 ln Q, Q = L(s+b) / L(b) for Poisson bins: -2 ln Q = 2 sum s_i - 2 X;
  larger X is more signal-like);
  CL_s+b = P_{s+b}(X <= X_obs), CL_b = P_b(X <= X_obs), CL_s = CL_s+b / CL_b,
  each P the fraction of toys.
"""
from __future__ import annotations

import math

import numpy as np

from .ipa_oracle import _philox_call, u01

PIECE = 400.0


def _uniform(i, k, h, m, seed):
    x = _philox_call(np.asarray([i], dtype=np.uint64), k, 8 + (h << 16) + (m >> 1), seed)
    w = 2 * (m & 1)
    return float(u01(x[w], x[w + 1])[0])


def poisson_piece(nu: float, u: float) -> int:
    n = 0
    p = math.exp(-nu)
    F = p
    cap = math.floor(nu + 40.0 * math.sqrt(nu) + 100.0)
    while u > F and p > 0.0 and n < cap:
        n += 1
        p = (p * nu) / n
        F = F + p
    return n


def poisson_bin(lam: float, i: int, k: int, h: int, seed: int) -> int:
    if not lam > 0.0:
        return 0
    M = max(1, math.ceil(lam / PIECE))
    nu = lam / M
    return sum(poisson_piece(nu, _uniform(i, k, h, m, seed)) for m in range(M))


def generate_binned(lam, seed: int, toy: int, hyp: int = 0) -> np.ndarray:
    """Counts of toy `toy` for bin means lam (plain loop over bins)."""
    lam = np.asarray(lam, dtype=np.float64)
    return np.array([poisson_bin(float(lam[i]), i, toy, hyp, seed) for i in range(lam.size)], dtype=np.int64)


def generate_binned_fast(lam, seed: int, toy: int, hyp: int = 0) -> np.ndarray:
    """The same counts, with the Philox calls of all bins drawn at once (the
    inversion itself still runs bin by bin).  Means above PIECE use the plain
    routine."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.size
    x = _philox_call(np.arange(n, dtype=np.uint64), toy, 8 + (hyp << 16), seed)
    u = u01(x[0], x[1])
    out = np.zeros(n, dtype=np.int64)
    for i in range(n):
        li = float(lam[i])
        if not li > 0.0:
            continue
        out[i] = poisson_piece(li, float(u[i])) if li <= PIECE else poisson_bin(li, i, toy, hyp, seed)
    return out


def smear(h, width: float, sigma: float) -> np.ndarray:
    h = np.asarray(h, dtype=np.float64)
    R = math.ceil(8.0 * sigma / width)
    d = np.arange(-R, R + 1)
    k = np.exp(-((d * width) ** 2) / (2.0 * sigma * sigma))
    k = k / math.fsum(k)
    n = h.size
    out = np.zeros(n)
    for i in range(n):
        lo, hi = max(0, i - R), min(n - 1, i + R)
        j = np.arange(lo, hi + 1)
        out[i] = math.fsum(k[i - j + R] * h[j])
    return out


def weights(s, b) -> np.ndarray:
    """w_i = ln(1 + s_i / b_i)."""
    return np.log1p(np.asarray(s, dtype=np.float64) / np.asarray(b, dtype=np.float64))


def statistic(counts, w) -> float:
    return math.fsum(np.asarray(counts, dtype=np.float64) * w)


def cls(s, b, data, n_toys: int, seed: int):
    """(CL_b, CL_s+b, CL_s), the counts of toys with X <= X_obs under b and s+b,
    and the statistics (X_b[k], X_sb[k], X_obs)."""
    s = np.asarray(s, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    w = weights(s, b)
    x_obs = statistic(data, w)
    lam_b, lam_sb = b, s + b
    xb = np.array([statistic(generate_binned_fast(lam_b, seed, k, 0), w) for k in range(n_toys)])
    xsb = np.array([statistic(generate_binned_fast(lam_sb, seed, k, 1), w) for k in range(n_toys)])
    nb = int(np.sum(xb <= x_obs))
    nsb = int(np.sum(xsb <= x_obs))
    cl_b, cl_sb = nb / n_toys, nsb / n_toys
    return (cl_b, cl_sb, cl_sb / cl_b if nb else math.nan), (nb, nsb), (xb, xsb, x_obs)
