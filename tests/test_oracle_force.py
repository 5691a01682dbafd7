"""Pins of the oracle's force term (Eq. F_def) and of its place in L (Eq. ecast)
against what the paper states it does (CPU only).

Sec. 2.5: taking the moments 1 and p of the Boltzmann equation gives
Eq. macro_u, rho (d_t u + u.grad u) = n F - grad p^i - div Pi, and the force
of Eq. F_def, F = grad(p^i - p^w)/n + sigma grad(Laplacian n), turns it into
Eq. macro_u_waals, where the ideal pressure p^i = n T is replaced by the van
der Waals pressure p^w of Eq. vdw and a capillary term n sigma grad(Laplacian n)
appears.  For a state at local equilibrium at rest, f = f^eq(n(x, y), 0,
T(x, y)), the viscous stress Pi and the velocity vanish, so the momentum
source of L is, to the truncation order of the stencils and fluxes,

    sum_kappa p_alpha L_kappa = -d_alpha p^w + n sigma d_alpha Laplacian(n).

The force enters L only through -F . grad_p f, and f, its fluxes and its
equilibrium do not depend on a, b or sigma.  The difference of L between the
van der Waals fluid and the ideal gas (a = b = sigma = 0, where F = 0) on the
same populations therefore isolates the force exactly:

    sum_kappa p_alpha (L - L_ideal)_kappa = n F_alpha
        = d_alpha (p^i - p^w) + n sigma d_alpha Laplacian(n),

to the 4th-order truncation of the 49-point stencils alone, while
sum_kappa p_alpha L_ideal_kappa = -d_alpha p^i to the accuracy of the WENO-5
fluxes.  Together they give the balance above.  Both sides are evaluated for
smooth periodic n and T, the right-hand sides with exact derivatives (sympy),
and F itself is checked against Eq. F_def.  The errors must be small and fall
at the order of the scheme when the grid is refined.

A test plants, one at a time, the mistakes that the other pins cannot see
(the force has no effect on the rest state, on mass conservation, on the
mirror tests or on a uniform-density shear wave) in a copy of the oracle and
checks that each one fails the pin."""
import math

import numpy as np
import pytest

import oracle
from paper_1702_01690_gb300 import inputs

sp = pytest.importorskip("sympy")

A, B = 9.0 / 8.0, 1.0 / 3.0   # Eq. vdw in the a/b form
SIGMA = 5e-3                   # large enough that the capillary term is ~half of the source


def exact_fields():
    """n, T (smooth, periodic on the unit square) and the exact right-hand
    sides: F of Eq. F_def and the momentum source of Eq. macro_u_waals."""
    x, y = sp.symbols("x y", real=True)
    tp = 2 * sp.pi
    n = sp.Rational(1, 2) + sp.Rational(8, 100) * sp.sin(tp * x) * sp.cos(tp * y) + sp.Rational(3, 100) * sp.cos(tp * (x + y) + 1)
    T = sp.Rational(13, 10) + sp.Rational(5, 100) * sp.cos(tp * x + sp.Rational(3, 10)) * sp.sin(tp * y + sp.Rational(7, 10))
    pi = n * T
    pw = n * T / (1 - B * n) - A * n ** 2
    lap = sp.diff(n, x, 2) + sp.diff(n, y, 2)
    out = {"n": n, "T": T}
    for ax, v in (("x", x), ("y", y)):
        out["F" + ax] = sp.diff(pi - pw, v) / n + SIGMA * sp.diff(lap, v)
        out["nF" + ax] = n * out["F" + ax]
        out["P" + ax] = -sp.diff(pi, v)
        out["M" + ax] = -sp.diff(pw, v) + n * SIGMA * sp.diff(lap, v)
    return {k: sp.lambdify((x, y), e, "numpy") for k, e in out.items()}, (x, y)


EXACT, _ = exact_fields()


def sampled(N):
    xs = inputs.node_x(N, 1.0 / N)
    X, Y = np.meshgrid(xs, xs)
    return {k: np.broadcast_to(np.asarray(f(X, Y), dtype=np.float64), X.shape).copy() for k, f in EXACT.items()}


def momentum_sources(N, a, b, sigma, ex, library=None):
    """L of f = f^eq(n, 0, T) on an N x N periodic grid, its momentum sources
    sum_kappa p L_kappa and the oracle's stage fields."""
    z = np.zeros((N, N))
    o = oracle.Oracle(N, N, 1.0 / N, 1e-4, 0.01, a, b, sigma, library=library)
    o.init_fields(ex["n"], z, z.copy(), ex["T"])
    ev = o.evaluate()
    o.close()
    R, _ = oracle.quadrature()
    L = ev["L"]
    return ev, sum(R[k // 5] * L[k] for k in range(25)), sum(R[k % 5] * L[k] for k in range(25))


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def force_errors(N, library=None):
    """Errors, relative to the largest exact value of each quantity, on an
    N x N grid: F against Eq. F_def (Fx, Fy), the force's momentum source
    n F (nFx, nFy), the ideal gas's momentum source against -grad p^i (Px,
    Py), the whole source against Eq. macro_u_waals (Mx, My), and the mass
    source sum_kappa L (relative to the momentum source's scale; 0 at rest)."""
    ex = sampled(N)
    ev, Mx, My = momentum_sources(N, A, B, SIGMA, ex, library)
    _, Px, Py = momentum_sources(N, 0.0, 0.0, 0.0, ex, library)
    err = {"Fx": rel(ev["Fx"], ex["Fx"]), "Fy": rel(ev["Fy"], ex["Fy"]),
           "nFx": rel(Mx - Px, ex["nFx"]), "nFy": rel(My - Py, ex["nFy"]),
           "Px": rel(Px, ex["Px"]), "Py": rel(Py, ex["Py"]),
           "Mx": rel(Mx, ex["Mx"]), "My": rel(My, ex["My"])}
    err["mass"] = float(np.max(np.abs(ev["L"].sum(axis=0))) / np.max(np.abs(ex["Mx"])))
    return err


FORCE_TOL = 2e-5   # F and n F at N = 64 (4th-order stencils)
FLUX_TOL = 1e-5    # -grad p^i and the whole balance at N = 64 (WENO-5-JS fluxes)


def test_force_matches_eq_F_def():
    """F of the oracle against Eq. F_def, and the momentum that the force term
    -F . grad_p f puts into L against n F: 4th order in ds."""
    e32, e64 = force_errors(32), force_errors(64)
    print("N=32", e32, "\nN=64", e64)
    for key in ("Fx", "Fy", "nFx", "nFy"):
        assert e64[key] < FORCE_TOL, (key, e64)
        order = math.log2(e32[key] / e64[key])
        assert order > 3.7, (key, order, e32, e64)


def test_force_replaces_ideal_pressure_by_vdw_pressure():
    """Eq. macro_u_waals at rest: the momentum source of L equals
    -grad p^w + n sigma grad(Laplacian n), and without the force (ideal gas)
    -grad p^i; both converge as the grid is refined.  Mass has no source."""
    e = {N: force_errors(N) for N in (32, 64, 128)}
    print(e)
    for key in ("Px", "Py", "Mx", "My"):
        assert e[64][key] < FLUX_TOL, (key, e[64])
        assert e[128][key] < e[64][key] / 8 < e[32][key] / 64, (key, e)
    assert e[64]["mass"] < FLUX_TOL


# Mistakes planted in a copy of the oracle's source; each must fail the pin.
PLANTED = {
    "force term with the wrong sign in L":
        ("double coll = (fq[kap] - feq[kap]) / p->tau;\n            c->L[(size_t)q * K + kap] = -advx - advy - force - coll;",
         "double coll = (fq[kap] - feq[kap]) / p->tau;\n            c->L[(size_t)q * K + kap] = -advx - advy + force - coll;"),
    "gradient-of-Laplacian divided by ds instead of ds^3":
        ("c->Fx[q] = (gx / ds) / c->n[q] + p->sigma * (lx / ds3);",
         "c->Fx[q] = (gx / ds) / c->n[q] + p->sigma * (lx / ds);"),
    "pressure term multiplied by n instead of divided":
        ("c->Fx[q] = (gx / ds) / c->n[q] + p->sigma * (lx / ds3);",
         "c->Fx[q] = (gx / ds) * c->n[q] + p->sigma * (lx / ds3);"),
    "capillary term with the wrong sign":
        ("c->Fy[q] = (gy / ds) / c->n[q] + p->sigma * (ly / ds3);",
         "c->Fy[q] = (gy / ds) / c->n[q] - p->sigma * (ly / ds3);"),
    "Delta p with p^i and p^w swapped":
        ("c->dp[q] = m4[0] * m4[3] - orc_pw(m4[0], m4[3], p->a, p->b);",
         "c->dp[q] = orc_pw(m4[0], m4[3], p->a, p->b) - m4[0] * m4[3];"),
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_planted_force_mistake_fails_the_pin(name, tmp_path):
    before, after = PLANTED[name]
    text = oracle.source()
    assert text.count(before) == 1, "the line to plant the mistake in has changed"
    lib = oracle.load_variant(text.replace(before, after), str(tmp_path))
    err = force_errors(64, library=lib)
    assert max(err[k] for k in ("Fx", "Fy", "nFx", "nFy")) > 100 * FORCE_TOL, err
