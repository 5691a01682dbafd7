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
