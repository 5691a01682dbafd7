"""The C-ABI library loads on a machine without a GPU, exports every function
include/olb.h declares, and rejects invalid parameters before touching the
device (CPU only)."""
import ctypes

import pytest

from helpers import header_functions


@pytest.fixture(scope="module")
def olb():
    from paper_1702_01690_gb300 import build
    build.build()
    from paper_1702_01690_gb300 import olb as mod
    return mod


def test_every_declared_symbol_is_exported(olb):
    names = header_functions()
    assert "olb_create" in names and "olb_step" in names
    lib = olb.library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(olb.SYMBOLS) == set(names)


def test_side_enum_matches_header(olb):
    import re
    from pathlib import Path
    text = (Path(__file__).resolve().parents[1] / "include" / "olb.h").read_text()
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"OLB_SIDE_(\w+) = (\d+)", text)}
    assert vals == {"PERIODIC": olb.SIDE_PERIODIC, "DIFFUSE": olb.SIDE_DIFFUSE, "SPECULAR": olb.SIDE_SPECULAR,
                    "SPECULAR_DIFFUSE": olb.SIDE_SPECULAR_DIFFUSE}


def test_params_struct_layout_matches_header(olb):
    # 2 ints, 6 doubles, 2+2 doubles, 4 ints (with natural alignment)
    assert ctypes.sizeof(olb.Params) == 8 + 6 * 8 + 4 * 8 + 4 * 4


def _params(olb, **kw):
    from paper_1702_01690_gb300 import inputs
    p, _ = inputs.planar_walls(nx=64, ny=8)
    pp = olb.params_from(p)
    for k, v in kw.items():
        if k in ("Tw", "uw"):
            getattr(pp, k)[0], getattr(pp, k)[1] = v
        else:
            setattr(pp, k, v)
    return pp


@pytest.mark.parametrize("kw,code", [
    (dict(nx=0), -1), (dict(ny=0), -1), (dict(nx=2), -1), (dict(ds=0.0), -1),
    (dict(dt=-1.0), -1), (dict(tau=0.0), -1), (dict(sigma=-1e-4), -1),
    (dict(side_x=7), -1), (dict(side_y=1), -1), (dict(precision=9), -1),
    (dict(weno_mode=3), -1), (dict(Tw=(0.0, 0.9)), -1), (dict(b=-0.1), -1),
    (dict(side_x=4), -1), (dict(side_y=3), -1), (dict(side_x=2, nx=2), -1), (dict(side_y=2, ny=2), -1),
    (dict(side_x=3, Tw=(0.9, 0.0)), -1),
    (dict(dt=1.0 / 64 / 2.8), -2), (dict(dt=0.1, ds=1.0), -2), (dict(dt=0.02, tau=0.005, ds=0.5), -2),
])
def test_create_rejects_invalid_params(olb, kw, code):
    pp = _params(olb, **kw)
    h = ctypes.c_void_p()
    assert olb.library().olb_create(ctypes.byref(pp), None, ctypes.byref(h)) == code
    assert not h.value


def test_null_arguments_rejected(olb):
    lib = olb.library()
    assert lib.olb_create(None, None, None) == -1
    assert lib.olb_step(None, 1) == -1
    assert lib.olb_moments(None, None, None, None, None) == -1
    assert lib.olb_get_populations(None, None) == -1
    lib.olb_destroy(None)


def test_status_strings(olb):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert olb.status_string(code).startswith("OLB_")
    assert "unknown" in olb.status_string(42)


def test_allocator_hook_needs_both_functions(olb):
    lib = olb.library()
    a = olb.ALLOC_FN(lambda n, s, u: None)
    assert lib.olb_set_allocator(a, olb.FREE_FN(0), None) == -1
    assert lib.olb_set_allocator(olb.ALLOC_FN(0), olb.FREE_FN(0), None) == 0
