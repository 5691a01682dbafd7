"""Closed-form van der Waals thermodynamics used as pins (test infrastructure).

p^w(n, T) = n T / (1 - b n) - a n^2 is Eq. vdw in the a/b form (a = 9/8,
b = 1/3 gives 3 n T / (3 - n) - 9/8 n^2, critical point n_c = T_c = 1).
The Maxwell equal-area construction (Sec. 4 and Sec. 4.4 of the paper)
gives the coexisting vapour / liquid densities: equal pressure and equal
chemical potential mu = T ln(n / (1 - b n)) + T b n / (1 - b n) - 2 a n,
which is the same as equal areas under p(v), v = 1/n.
"""
from __future__ import annotations

import math

A_VDW = 9.0 / 8.0
B_VDW = 1.0 / 3.0


def pressure(n: float, T: float, a: float = A_VDW, b: float = B_VDW) -> float:
    return n * T / (1.0 - b * n) - a * n * n


def chem_potential(n: float, T: float, a: float = A_VDW, b: float = B_VDW) -> float:
    return T * math.log(n / (1.0 - b * n)) + T * b * n / (1.0 - b * n) - 2.0 * a * n


def spinodal(T: float, a: float = A_VDW, b: float = B_VDW):
    """Densities where dp/dn = T / (1 - b n)^2 - 2 a n vanishes."""
    def dp(n):
        return T / (1.0 - b * n) ** 2 - 2.0 * a * n
    nc = 1.0 / (3.0 * b)
    lo = _bisect(dp, 1e-12, nc)
    hi = _bisect(dp, nc, (1.0 - 1e-12) / b)
    return lo, hi


def _bisect(fn, lo, hi, iters=200):
    flo = fn(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = fn(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def coexistence(T: float, a: float = A_VDW, b: float = B_VDW):
    """(n_gas, n_liquid) at temperature T < T_c by Newton's method on
    p(n_g) = p(n_l), mu(n_g) = mu(n_l), started inside the spinodal branches."""
    s_lo, s_hi = spinodal(T, a, b)
    ng, nl = 0.5 * s_lo, min(0.5 * (s_hi + 1.0 / b), s_hi * 1.3)
    for _ in range(200):
        F1 = pressure(ng, T, a, b) - pressure(nl, T, a, b)
        F2 = chem_potential(ng, T, a, b) - chem_potential(nl, T, a, b)
        dpg = T / (1.0 - b * ng) ** 2 - 2.0 * a * ng
        dpl = T / (1.0 - b * nl) ** 2 - 2.0 * a * nl
        # d mu / d n = (dp/dn) / n
        J = [[dpg, -dpl], [dpg / ng, -dpl / nl]]
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0]
        dng = (F1 * J[1][1] - F2 * J[0][1]) / det
        dnl = (J[0][0] * F2 - J[1][0] * F1) / det
        step = 1.0
        while True:
            ng_new, nl_new = ng - step * dng, nl - step * dnl
            if 0.0 < ng_new < s_lo and s_hi < nl_new < 1.0 / b:
                break
            step *= 0.5
        ng, nl = ng_new, nl_new
        if abs(dng) < 1e-16 and abs(dnl) < 1e-16:
            break
    return ng, nl


def interface_width(sigma: float, Tw: float) -> float:
    """xi_w = sqrt(8 sigma / (9 (1 - T_w))) (Eq. xiwagner, reading kappa as
    the surface-tension parameter sigma)."""
    return math.sqrt(8.0 * sigma / (9.0 * (1.0 - Tw)))
