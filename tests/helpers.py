"""Shared test utilities (comparison norms, oracle set-up, window crops)."""
import re
import os

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    """Names of the functions that include/*.h declares."""
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(olb_\w+)\s*\(", txt)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def field_rel(a, b):
    """max |a - b| / max |b|: error relative to the field's magnitude."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0))


def moments_rel(m_gpu, m_ref):
    """Errors of (n, u, T) relative to each field's magnitude; u_x and u_y
    share the scale max(|u_x|, |u_y|) since one of them may be ~0."""
    n1, ux1, uy1, T1 = m_gpu
    n0, ux0, uy0, T0 = m_ref
    us = max(np.max(np.abs(ux0)), np.max(np.abs(uy0)), 1e-300)
    return {
        "n": field_rel(n1, n0),
        "u": float(max(np.max(np.abs(ux1 - ux0)), np.max(np.abs(uy1 - uy0))) / us),
        "T": field_rel(T1, T0),
    }


def make_oracle(p, fields):
    o = oracle.Oracle(p.nx, p.ny, p.ds, p.dt, p.tau, p.a, p.b, p.sigma, p.Tw, p.uw, p.side_x, p.side_y)
    o.init_fields(*fields)
    return o


EPS = float(np.finfo(np.float64).eps)


def rounding_envelope(p, fields, steps, ulps=4.0, seed=0):
    """How far two correct FP64 evaluations of the same run can drift apart.

    The step is ill-conditioned where the 49-point stencils of Eq. F_def
    cancel to O(ds^k) of their terms (fine grids, smooth fields): a 1-ulp
    change of the state moves the force by up to ~1e6 ulp.  The oracle is run
    twice, the second time with every population multiplied by
    1 + ulps * eps * U(-1, 1) before each step, a stand-in for the rounding
    of one RK-3 step done in another order.  The absolute differences of
    (n, u_x, u_y, T) between the two runs and the unperturbed oracle are
    returned; callers bound errors by the maximum of a difference over the
    compared region (pointwise, a random perturbation can happen to cancel)."""
    a = make_oracle(p, fields)
    b = make_oracle(p, fields)
    rng = np.random.default_rng(seed)
    for _ in range(steps):
        f = b.get_populations()
        b.set_populations(f * (1.0 + ulps * EPS * rng.uniform(-1.0, 1.0, f.shape)))
        a.step(1)
        b.step(1)
    return [np.abs(x - y) for x, y in zip(a.moments(), b.moments())], a


def check_against_envelope(m_gpu, p, fields, steps, rtol=1e-11, factor=10.0):
    """GPU moments vs the oracle: each field within max(rtol x its magnitude,
    factor x the largest spread of the rounding envelope over the grid).
    Returns the worst ratio error / allowed (< 1 passes) per field."""
    env, o = rounding_envelope(p, fields, steps)
    ref = o.moments()
    us = max(np.max(np.abs(ref[1])), np.max(np.abs(ref[2])), 1e-300)
    scales = [np.max(np.abs(ref[0])), us, us, np.max(np.abs(ref[3]))]
    out = {}
    for name, g, r, e, s in zip(("n", "ux", "uy", "T"), m_gpu, ref, env, scales):
        allowed = max(rtol * s, factor * float(np.max(e)))
        out[name] = float(np.max(np.abs(np.asarray(g) - r) / allowed))
    return out


def symmetric_fields(nx, ny, sym_x, sym_y, seed):
    """Smooth random fields, even (n, T, the tangential velocity) or odd (the
    normal velocity) under i -> nx-1-i (sym_x) and j -> ny-1-j (sym_y)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)

    def smooth(amp):
        a = rng.uniform(-1, 1, 4)
        return amp * (a[0] * np.cos(2 * np.pi * X + a[1]) * np.cos(2 * np.pi * Y + a[2])
                      + a[3] * np.sin(4 * np.pi * X + a[2]) * np.sin(2 * np.pi * Y + a[1]))

    n = 1.0 + smooth(0.05)
    ux, uy = smooth(0.02), smooth(0.02)
    T = 0.95 + smooth(0.02)
    if sym_x:
        n, T, uy = [(v + v[:, ::-1]) / 2 for v in (n, T, uy)]
        ux = (ux - ux[:, ::-1]) / 2
    if sym_y:
        n, T, ux = [(v + v[::-1, :]) / 2 for v in (n, T, ux)]
        uy = (uy - uy[::-1, :]) / 2
    return n, ux, uy, T
