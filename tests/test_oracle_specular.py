"""Pins of the oracle's specular sides (Sec. 3.4.1) and the field double
reflection at corners (Sec. 3.4.3), CPU only.

A state that is mirror-symmetric about a plane stays symmetric, so a run on
the reduced domain with specular reflection on that plane must reproduce
the full-domain run (which uses no specular code) on the kept part.  A wrong
velocity reflection, ghost offset, field reflection or corner rule changes
the reduced run at first order."""
import numpy as np
import pytest

import oracle
from helpers import symmetric_fields

TOL = 1e-12


def run(nx, ny, fields, steps, side_x, side_y, ds, dt=2e-4):
    o = oracle.Oracle(nx, ny, ds, dt, 0.005, sigma=1e-4, Tw=(0.9, 0.9), side_x=side_x, side_y=side_y)
    o.init_fields(*fields)
    o.step(steps)
    return o.get_populations(), o


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_half_channel_equals_full_channel():
    """Diffuse walls at x = 0, 1 (full) vs specular x = 1/2 and the wall at
    x = 1 (the paper's half channel, Sec. 4)."""
    M, ny = 12, 5
    fl = symmetric_fields(2 * M, ny, True, False, 1)
    full, _ = run(2 * M, ny, fl, 4, 1, 0, 1.0 / (2 * M))
    half, _ = run(M, ny, [v[:, M:] for v in fl], 4, 3, 0, 1.0 / (2 * M))
    assert rel(half, full[:, :, M:]) < TOL


def test_specular_x_sides_equal_periodic_symmetric_state():
    """Periodic x, state even about x = 1/2 (and so about x = 0): the first
    half with specular x sides reproduces it."""
    M, ny = 9, 4
    fl = symmetric_fields(2 * M, ny, True, False, 2)
    full, _ = run(2 * M, ny, fl, 4, 0, 0, 1.0 / (2 * M))
    half, _ = run(M, ny, [v[:, :M] for v in fl], 4, 2, 0, 1.0 / (2 * M))
    assert rel(half, full[:, :, :M]) < TOL


def test_specular_y_sides_equal_periodic_symmetric_state():
    """Periodic y, state even about y = 1/2: the lower half with specular y
    sides reproduces it (y ghosts reverse k2)."""
    nx, M = 7, 6
    fl = symmetric_fields(nx, 2 * M, False, True, 3)
    full, _ = run(nx, 2 * M, fl, 4, 0, 0, 1.0 / (2 * M))
    half, _ = run(nx, M, [v[:M, :] for v in fl], 4, 0, 2, 1.0 / (2 * M))
    assert rel(half, full[:, :M, :]) < TOL


def test_quarter_domain_equals_full_domain():
    """The paper's reduced Laplace domain (Sec. 5): specular bottom, left and
    top, diffuse wall on the right; corners take the double field
    reflection.  Full domain: walls at x = 0, 1, periodic y, state even about
    x = 1/2 and y = 1/2."""
    M = 8
    fl = symmetric_fields(2 * M, 2 * M, True, True, 4)
    full, _ = run(2 * M, 2 * M, fl, 4, 1, 0, 1.0 / (2 * M))
    quarter, _ = run(M, M, [v[:M, M:] for v in fl], 4, 3, 2, 1.0 / (2 * M))
    assert rel(quarter, full[:, :M, M:]) < TOL


def test_specular_box_conserves_mass_and_is_closed():
    """Specular sides on all four sides: no mass crosses a mirror plane."""
    fl = symmetric_fields(10, 8, False, False, 5)
    o = oracle.Oracle(10, 8, 0.1, 2e-3, 0.005, sigma=1e-4, side_x=2, side_y=2)
    o.init_fields(*fl)
    m0 = o.moments()[0].sum()
    o.step(50)
    assert abs(o.moments()[0].sum() - m0) < 1e-13 * m0


@pytest.mark.parametrize("nx,ny,sx,sy", [(2, 5, 2, 0), (5, 2, 0, 2), (6, 6, 4, 0), (6, 6, 0, 1), (2, 4, 3, 0)])
def test_invalid_specular_configurations_rejected(nx, ny, sx, sy):
    with pytest.raises(ValueError):
        oracle.Oracle(nx, ny, 0.1, 1e-3, 0.01, side_x=sx, side_y=sy)
