"""Pins of the FP64 oracle's building blocks against what the paper and the
mathematics fix (closed forms, printed values, library routines, brute force).

Every test here runs on the CPU."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import hermite_e as HE

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def frac(s):
    return float(Fraction(s))


# ------------------------------------------------------------ quadrature

def test_quadrature_matches_library_gauss_hermite():
    """Table trots against numpy's probabilists' Gauss-Hermite rule."""
    R, W = oracle.quadrature()
    x, w = HE.hermegauss(5)
    np.testing.assert_allclose(R, x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(W, w / math.sqrt(2 * math.pi), rtol=1e-14)
    assert abs(W.sum() - 1.0) < 1e-15


def test_quadrature_roots_and_weight_formula():
    """He_5(R_q) = 0 and W_q = Q!/He_6(R_q)^2 (Sec. 2.2), with He from numpy."""
    R, W = oracle.quadrature()
    he5 = HE.hermeval(R, [0] * 5 + [1])
    he6 = HE.hermeval(R, [0] * 6 + [1])
    assert np.max(np.abs(he5)) < 1e-12
    np.testing.assert_allclose(W, 120.0 / he6 ** 2, rtol=1e-13)
    assert abs(R[-1] - GOLD["quadrature"]["p_max_approx"]) < 0.005


def test_hermite_matches_numpy():
    rng = np.random.default_rng(1)
    for l in range(8):
        for x in rng.uniform(-3, 3, 5):
            ref = HE.hermeval(x, [0] * l + [1])
            assert abs(oracle.hermite(l, x) - ref) <= 1e-12 * max(1.0, abs(ref))


# ------------------------------------------------------------ equilibrium

def gaussian_moment(m, u, T):
    """E[(u + sqrt(T) Z)^m], Z standard normal."""
    return sum(math.comb(m, 2 * s) * u ** (m - 2 * s) * T ** s * math.prod(range(1, 2 * s, 2))
               for s in range(m // 2 + 1))


@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.3, 0.8), (-0.7, 1.3), (1.5, 0.5), (0.05, 2.0)])
def test_g_reproduces_gaussian_moments_to_order_4(u, T):
    """Eq. g_alpha: sum_k g_k(u,T) p_k^m is the m-th moment of a Maxwellian of
    velocity u and temperature T (m = 1) for m = 0..4; order 5 is not."""
    R, _ = oracle.quadrature()
    g = np.array([oracle.g(k, u, T) for k in range(5)])
    for m in range(5):
        ref = gaussian_moment(m, u, T)
        assert abs((g * R ** m).sum() - ref) < 1e-13 * max(1.0, abs(ref))
    if abs(u) > 0.1:
        assert abs((g * R ** 5).sum() - gaussian_moment(5, u, T)) > 1e-6


def test_feq_moments_2d():
    """Eq. feq: product form gives the 2-D Maxwellian moments."""
    R, _ = oracle.quadrature()
    px = np.repeat(R, 5)
    py = np.tile(R, 5)
    n, ux, uy, T = 1.7, 0.2, -0.35, 0.85
    f = oracle.feq(n, ux, uy, T)
    assert abs(f.sum() - n) < 1e-14
    assert abs((px * f).sum() - n * ux) < 1e-14
    assert abs((py * f).sum() - n * uy) < 1e-14
    assert abs((px * py * f).sum() - n * ux * uy) < 1e-14
    assert abs(((px ** 2 + py ** 2) * f).sum() - n * (ux * ux + uy * uy + 2 * T)) < 1e-13
    assert abs((px ** 2 * py ** 2 * f).sum() - n * (ux ** 2 + T) * (uy ** 2 + T)) < 1e-13


@pytest.mark.parametrize("state", [(1.0, 0.0, 0.0, 1.0), (0.24, 0.1, -0.2, 0.8),
                                   (1.93, -0.3, 0.05, 0.7), (0.5, 1.2, 0.9, 1.6)])
def test_moments_recover_equilibrium_state(state):
    """Moments (Sec. 2.2, T from the trace of Eq. sigmaq_def) of f^eq give back
    (n, u, T): pins the T-recovery reading together with Eq. feq."""
    f = oracle.feq(*state)
    np.testing.assert_allclose(oracle.moments_node(f), state, rtol=1e-13, atol=1e-14)


def test_collision_conserves_mass_momentum_energy():
    """f - f^eq(moments(f)) has zero mass, momentum and energy moments."""
    R, _ = oracle.quadrature()
    px = np.repeat(R, 5)
    py = np.tile(R, 5)
    rng = np.random.default_rng(7)
    for _ in range(5):
        f = oracle.feq(1.1, 0.1, -0.05, 0.9) * (1 + 0.2 * rng.uniform(-1, 1, 25))
        n, ux, uy, T = oracle.moments_node(f)
        d = f - oracle.feq(n, ux, uy, T)
        for wgt in (np.ones(25), px, py, px ** 2 + py ** 2):
            assert abs((wgt * d).sum()) < 1e-14 * n


# ------------------------------------------------------------ momentum derivative

def test_dp_line_is_exact_derivative_of_weighted_cubic():
    """Eq. derf: for f_k = w_k P(p_k) with P of degree <= 3 the truncated
    Hermite series is exact, so (d_p f)_k = w_k (P'(p_k) - p_k P(p_k))
    (derivative of omega(p) P(p) divided by omega)."""
    R, W = oracle.quadrature()
    rng = np.random.default_rng(3)
    for _ in range(10):
        c = rng.normal(size=4)
        P = np.polynomial.Polynomial(c)
        out = oracle.dp_line(W * P(R))
        ref = W * (P.deriv()(R) - R * P(R))
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13 * np.abs(c).max())


def test_dp_line_moment_sources():
    """sum_k (d_p f)_k = 0 (mass), sum_k p_k (d_p f)_k = -sum f (force n F),
    sum_k p_k^2 (d_p f)_k = -2 sum p f (work)."""
    R, _ = oracle.quadrature()
    rng = np.random.default_rng(4)
    for _ in range(10):
        f = rng.uniform(0.1, 1.0, 5)
        d = oracle.dp_line(f)
        assert abs(d.sum()) < 1e-14
        assert abs((R * d).sum() + f.sum()) < 1e-14
        assert abs((R ** 2 * d).sum() + 2 * (R * f).sum()) < 1e-13


# ------------------------------------------------------------ 49-point stencils

def apply_stencil(C, fn, h, power, x0=0.37, y0=-0.21):
    """sum_{l,m} C[m+3, l+3] fn(x0 + l h, y0 + m h) / h^power."""
    acc = 0.0
    for m in range(-3, 4):
        for l in range(-3, 4):
            acc += C[m + 3, l + 3] * fn(x0 + l * h, y0 + m * h)
    return acc / h ** power


def monomial(a, b):
    return lambda x, y: x ** a * y ** b


def d_dx(a, b, x, y):
    return a * x ** (a - 1) * y ** b if a > 0 else 0.0


def d_dx_lap(a, b, x, y):
    """d/dx of the Laplacian of x^a y^b."""
    t = 0.0
    if a >= 3:
        t += a * (a - 1) * (a - 2) * x ** (a - 3) * y ** b
    if a >= 1 and b >= 2:
        t += a * b * (b - 1) * x ** (a - 1) * y ** (b - 2)
    return t


@pytest.mark.parametrize("deg", range(0, 7))
def test_grad_stencil_exact_to_degree_6(deg):
    """Eq. stencil_grad is exact for every polynomial of degree <= 6 (6th order)."""
    C = oracle.grad_stencil()
    Cy = C.T
    h = 0.125
    for a in range(deg + 1):
        b = deg - a
        gx = apply_stencil(C, monomial(a, b), h, 1)
        gy = apply_stencil(Cy, monomial(a, b), h, 1)
        assert abs(gx - d_dx(a, b, 0.37, -0.21)) < 1e-11
        assert abs(gy - d_dx(b, a, -0.21, 0.37)) < 1e-11


def test_grad_stencil_not_exact_at_degree_7():
    C = oracle.grad_stencil()
    h = 0.125
    assert abs(apply_stencil(C, monomial(7, 0), h, 1) - d_dx(7, 0, 0.37, -0.21)) > 1e-9


def test_grad_stencil_1d_reduction_matches_paper():
    C = oracle.grad_stencil()
    g = GOLD["grad_stencil_1d"]
    col = C.sum(axis=0)  # sum over m at each l
    for off, cf in zip(g["offsets"], g["coefficients"]):
        assert abs(col[off + 3] - frac(cf)) < 1e-15


@pytest.mark.parametrize("deg", range(0, 7))
def test_glap_stencil_exact_to_degree_6(deg):
    """Eq. stencil_glap (with reading R1) is exact for degree <= 6 (4th order)."""
    C = oracle.glap_stencil()
    Cy = C.T
    h = 0.125
    for a in range(deg + 1):
        b = deg - a
        gx = apply_stencil(C, monomial(a, b), h, 3)
        gy = apply_stencil(Cy, monomial(a, b), h, 3)
        assert abs(gx - d_dx_lap(a, b, 0.37, -0.21)) < 1e-9
        assert abs(gy - d_dx_lap(b, a, -0.21, 0.37)) < 1e-9


def test_glap_stencil_1d_reduction_matches_paper():
    C = oracle.glap_stencil()
    g = GOLD["glap_stencil_1d"]
    col = C.sum(axis=0)
    for off, cf in zip(g["offsets"], g["coefficients"]):
        assert abs(col[off + 3] - frac(cf)) < 1e-14


def test_glap_printed_coefficients_are_inconsistent():
    """Reading R1: with c1, c4 as printed the 1-D reduction of Sec. 4 fails at
    offset 3, while the other printed coefficients agree with the oracle."""
    pc = GOLD["glap_printed_coefficients"]
    C = oracle.glap_stencil()
    # oracle keeps the printed c6..c12: entry (|m|=2,|l|=2) is c6 etc.
    assert abs(C[3 + 2, 3 + 2] - frac(pc["c6"])) < 1e-16
    assert abs(C[3 + 1, 3 + 2] - frac(pc["c7"])) < 1e-16
    assert abs(C[3 + 0, 3 + 2] - frac(pc["c8"])) < 1e-16
    assert abs(C[3 + 2, 3 + 1] - frac(pc["c10"])) < 1e-16
    assert abs(C[3 + 1, 3 + 1] - frac(pc["c11"])) < 1e-16
    assert abs(C[3 + 0, 3 + 1] - frac(pc["c12"])) < 1e-16
    printed_sum = 2 * frac(pc["c1"]) + frac(pc["c4"])
    assert abs(printed_sum - (-1 / 8)) > 0.1
    assert abs(2 * C[0, 6] + C[3, 6] - (-1 / 8)) < 1e-15


# ------------------------------------------------------------ WENO-5

def _table():
    return {tuple(r["zero"]): [frac(x) for x in r["w"]] for r in GOLD["weno_table"]["rows"]}


@pytest.mark.parametrize("v,zero", [
    ([2.0, 2.0, 2.0, 2.0, 2.0], (1, 2, 3)),
    ([1.3, 2.0, 2.0, 2.0, 2.0], (2, 3)),
    ([2.0, 2.0, 2.0, 2.0, 0.4], (1, 2)),
    ([2.0, 2.0, 2.0, 1.1, 0.3], (1,)),
    ([0.2, 2.0, 2.0, 2.0, 0.1], (2,)),
    ([0.7, 1.5, 2.0, 2.0, 2.0], (3,)),
])
def test_weno_table_rows(v, zero):
    """Table tab:weno for every pattern of vanishing indicators that data can
    produce (sigma_1 = sigma_3 = 0 forces all five values equal, hence
    sigma_2 = 0 too, so the (1/4, 0, 3/4) row is never reached)."""
    _, w = oracle.weno5(v, return_weights=True)
    np.testing.assert_allclose(w, _table()[zero], rtol=0, atol=1e-15)


def test_weno_ideal_weights_for_smooth_data():
    """With all indicators positive and equal the weights are delta."""
    h = 1e-3
    x = np.arange(-2, 3) * h
    _, w = oracle.weno5(np.sin(1.0 + x), return_weights=True)
    np.testing.assert_allclose(w, [0.1, 0.6, 0.3], atol=2e-3)


def test_weno_exact_derivative_for_quadratics():
    """For point values of a quadratic every candidate reconstructs the same
    interface value, so (F_{i+1/2} - F_{i-1/2})/h = f'(x_i) whatever the weights."""
    rng = np.random.default_rng(5)
    h = 0.1
    for _ in range(20):
        c = rng.normal(size=3)
        P = np.polynomial.Polynomial(c)
        xi = rng.uniform(-1, 1)
        xs = xi + h * np.arange(-3, 4)
        fv = P(xs)
        Fp = oracle.weno5(fv[1:6])   # face i+1/2 uses i-2..i+2
        Fm = oracle.weno5(fv[0:5])   # face i-1/2 uses i-3..i+1
        assert abs((Fp - Fm) / h - P.deriv()(xi)) < 1e-11 * max(1, np.abs(c).max())


def test_weno_fifth_order_on_smooth_function():
    """The derivative from WENO-5 fluxes converges at 5th order on a smooth
    periodic function (Sec. 3.2: fifth order for smooth functions)."""
    errs = []
    for N in (20, 40, 80):
        h = 1.0 / N
        x = np.arange(N) * h
        f = 2.0 + np.sin(2 * np.pi * x)
        ext = np.concatenate([f[-3:], f, f[:3]])
        F = np.array([oracle.weno5(ext[i:i + 5]) for i in range(N + 1)])  # face i-1/2
        d = (F[1:] - F[:-1]) / h
        errs.append(np.max(np.abs(d - 2 * np.pi * np.cos(2 * np.pi * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.5, (errs, orders)


def test_weno_scale_and_shift_invariant_weights():
    rng = np.random.default_rng(6)
    for _ in range(10):
        v = rng.uniform(0, 1, 5)
        _, w1 = oracle.weno5(v, return_weights=True)
        _, w2 = oracle.weno5(3.5 * v + 0.25, return_weights=True)
        np.testing.assert_allclose(w1, w2, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------ pressure / Maxwell

def test_vdw_general_form_is_eq_vdw():
    for n in (0.2, 1.0, 1.9):
        for T in (0.7, 1.0, 1.2):
            assert abs(oracle.pw(n, T, 9 / 8, 1 / 3) - (3 * n * T / (3 - n) - 9 / 8 * n * n)) < 1e-14


def test_vdw_critical_point():
    """p^w has an inflection with zero slope at n_c = T_c = 1, p_c = 3/8."""
    g = GOLD["vdw_critical_point"]
    h = 1e-4
    p = lambda n: oracle.pw(n, 1.0, 9 / 8, 1 / 3)
    assert abs(p(1.0) - g["p_c"]) < 1e-15
    assert abs((p(1 + h) - p(1 - h)) / (2 * h)) < 1e-7
    assert abs((p(1 + h) - 2 * p(1) + p(1 - h)) / h ** 2) < 1e-5


def test_maxwell_construction_matches_paper_T08():
    from oracle import maxwell
    from scipy.integrate import quad
    g = GOLD["maxwell_T08"]
    ng, nl = maxwell.coexistence(0.8)
    assert abs(ng - g["n_gas"]) < 1e-7
    assert abs(nl - g["n_liquid"]) < 5e-6
    # equal areas under p(v), v = 1/n, by quadrature
    ps = maxwell.pressure(ng, 0.8)
    area, _ = quad(lambda v: maxwell.pressure(1 / v, 0.8), 1 / nl, 1 / ng, epsabs=1e-13)
    assert abs(area - ps * (1 / ng - 1 / nl)) < 1e-10
    lo, hi = maxwell.spinodal(0.8)
    assert abs(lo - GOLD["spinodal_T08"]["n_low"]) < 1e-3
    assert abs(hi - GOLD["spinodal_T08"]["n_high"]) < 1e-3
