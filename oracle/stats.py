"""Integrated autocorrelation time and effective sample size.  TEST INFRASTRUCTURE ONLY.

Not part of arXiv:2011.12453; used to compare proposals.  Sokal's automatic
windowing (A. Sokal, "Monte Carlo methods in statistical mechanics: foundations and
new algorithms", 1997): tau(M) = 1 + 2 sum_{t=1}^{M} rho(t), with the window M the
smallest integer such that M >= c * tau(M), c = 5.
"""
from __future__ import annotations

import numpy as np


def rho(x: np.ndarray, t: int) -> float:
    """Normalised autocorrelation at lag t of a 1-D series (direct sum)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    d = x - x.mean()
    var = (d * d).sum() / n
    if var == 0.0:
        return 1.0 if t == 0 else 0.0
    return float((d[: n - t] * d[t:]).sum() / n / var)


def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    x = np.asarray(x, dtype=np.float64)
    tau = 1.0
    acc = 0.0
    for M in range(1, x.size):
        acc += rho(x, M)
        tau = 1.0 + 2.0 * acc
        if M >= c * tau:
            break
    return float(tau)


def ess(series_per_chain: np.ndarray) -> float:
    """Sum over chains of n / tau_int for a (C, n) array of per-chain series."""
    s = np.atleast_2d(series_per_chain)
    return float(sum(s.shape[1] / max(tau_int(row), 1e-12) for row in s))
