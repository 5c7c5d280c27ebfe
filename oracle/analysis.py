"""Integrated autocorrelation time, oracle side (plain numpy).

TEST INFRASTRUCTURE ONLY (see the oracle package header).

tau_int = 1/2 + sum_{t=1}^{W} rho(t) with Sokal's automatic window: the
smallest W with W >= c * tau_int(W), c = 5 (A. Sokal, "Monte Carlo methods in
statistical mechanics", 1996 lecture notes).  The effective sample count is
n / (2 tau_int).
"""
from __future__ import annotations

import numpy as np


def autocorr(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, float)
    n = len(x)
    d = x - x.mean()
    var = np.dot(d, d) / n
    if var == 0:
        return np.ones(1)
    return np.array([np.dot(d[: n - t], d[t:]) / (n * var) for t in range(n)])


def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    rho = autocorr(x)
    tau = 0.5
    for W in range(1, len(rho)):
        tau += rho[W]
        if W >= c * tau:
            return max(tau, 0.5)
    return max(tau, 0.5)
