"""Bernstein polynomial basis of the trajectory parametrisation, Eq. (param).

x(t_i) = W[i] . c_x, y(t_i) = W[i] . c_y, with derivatives through Wd, Wdd.
The paper states only "a 10th order polynomial" (Sec. V-A); this reference
uses the Bernstein form of degree n-1 on the grid tau_i = i / (m - 1),
t_i = i * dt, so t_f = (m - 1) * dt and d/dt = (1 / t_f) d/dtau.
"""
from __future__ import annotations

from math import comb

import numpy as np


def _bernstein(deg: int, k: int, tau: np.ndarray) -> np.ndarray:
    """b_{k,deg}(tau) = C(deg, k) tau^k (1 - tau)^(deg - k); zero outside 0..deg."""
    if k < 0 or k > deg:
        return np.zeros_like(tau)
    return comb(deg, k) * tau ** k * (1.0 - tau) ** (deg - k)


def bernstein(m: int, n: int, dt: float):
    """Return (W, Wd, Wdd), each (m, n) float64, for degree n-1.

    Derivatives use d/dtau b_{k,d} = d (b_{k-1,d-1} - b_{k,d-1}) applied once
    and twice, scaled by 1/t_f and 1/t_f^2.
    """
    deg = n - 1
    tf = (m - 1) * dt
    tau = np.arange(m, dtype=np.float64) / (m - 1)
    W = np.stack([_bernstein(deg, k, tau) for k in range(n)], axis=1)
    dW = np.stack([deg * (_bernstein(deg - 1, k - 1, tau) - _bernstein(deg - 1, k, tau))
                   for k in range(n)], axis=1)
    ddW = np.stack([deg * (deg - 1) * (_bernstein(deg - 2, k - 2, tau)
                                       - 2.0 * _bernstein(deg - 2, k - 1, tau)
                                       + _bernstein(deg - 2, k, tau))
                    for k in range(n)], axis=1)
    return W, dW / tf, ddW / tf ** 2
