"""Linearised hydrodynamic laws used as pins (test infrastructure).

Shear-wave damping (Sec. 6.1, Eq. shear_sol): u_y = u0 exp(-nu t) sin(k x)
with nu = k^2 eta_0 / rho_0 and eta_0 = tau n_0 T_0 (Chapman-Enskog, Sec. 2.4),
rho_0 = m n_0 with m = 1, so nu = k^2 tau T_0.
"""
from __future__ import annotations

import math

import numpy as np


def shear_decay_rate(k: float, tau: float, T0: float) -> float:
    return k * k * tau * T0


def shear_amplitude(uy: np.ndarray, x: np.ndarray, k: float) -> float:
    """Discrete projection (2/N) sum_i u_y,i sin(k x_i) (Sec. 6.1),
    averaged over rows."""
    uy = np.asarray(uy, dtype=np.float64)
    s = np.sin(k * np.asarray(x, dtype=np.float64))
    return float(2.0 / uy.shape[-1] * np.mean(uy @ s if uy.ndim > 1 else uy @ s))
