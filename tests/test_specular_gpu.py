"""Specular sides (Sec. 3.4.1) on the CUDA path: parity with the FP64 oracle,
shape independence, reduced domains against full mirror-symmetric ones,
FP32 and batches (GPU)."""
import numpy as np
import pytest

from helpers import field_rel, make_oracle, moments_rel, symmetric_fields
from paper_1702_01690_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
CONFIGS = [(2, 0), (3, 0), (0, 2), (2, 2), (3, 2)]


@pytest.fixture(scope="module")
def olb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01690_gb300 import build
    build.build()
    from paper_1702_01690_gb300 import olb as mod
    return mod


def setup(nx, ny, side_x, side_y, seed=9):
    p = inputs.RunParams(nx=nx, ny=ny, ds=1.0 / nx, dt=0.2 / nx / inputs.P_MAX, tau=0.01,
                         Tw=(0.85, 0.95), side_x=side_x, side_y=side_y)
    n, ux, uy, T = inputs.noisy_rest(nx, ny, seed, 1.0, 0.05, 1.0)
    rng = np.random.default_rng(seed + 1)
    ux = 0.01 * rng.uniform(-1, 1, n.shape)
    uy = 0.01 * rng.uniform(-1, 1, n.shape)
    return p, (n, ux, uy, T)


@pytest.mark.parametrize("nx,ny", [(45, 19), (12, 5)])
@pytest.mark.parametrize("sides", CONFIGS)
def test_specular_matches_oracle(olb, sides, nx, ny):
    """Populations and moments after 4 steps against the oracle, on a grid
    with ragged tiles (45 x 19) and one smaller than a tile (12 x 5)."""
    p, fl = setup(nx, ny, *sides)
    ctx = olb.create(p)
    ctx.init_fields(*fl)
    o = make_oracle(p, fl)
    assert ctx.step(4) == 0
    o.step(4)
    assert field_rel(ctx.get_populations(), o.get_populations()) < FP64_TOL
    assert max(moments_rel(ctx.moments(), o.moments()).values()) < FP64_TOL


def test_every_tile_shape_identical_with_specular_sides(olb):
    p, fl = setup(45, 19, 3, 2)
    ref = None
    for shape in ((8, 8, 4), (16, 8, 2), (16, 8, 1), (32, 8, 1), (32, 16, 1), (8, 8, 8), (7, 8, 8), (8, 8, 5)):
        ctx = olb.create(p)
        ctx.set_tile(*shape)
        ctx.init_fields(*fl)
        assert ctx.step(4) == 0
        f = ctx.get_populations()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref), shape


def test_reduced_laplace_domain_equals_full_domain(olb):
    """The paper's reduced Laplace domain (Sec. 5: specular bottom, left and
    top, diffuse wall on the right) on the GPU reproduces the full domain
    (walls at x = 0, 1, periodic y) started from a state even about x = 1/2
    and y = 1/2, over 20 steps."""
    M = 40
    fl = symmetric_fields(2 * M, 2 * M, True, True, 11)
    kw = dict(ds=1.0 / (2 * M), dt=2e-4 * 160 / (2 * M), tau=0.005, Tw=(0.9, 0.9))
    full = olb.create(inputs.RunParams(nx=2 * M, ny=2 * M, side_x=1, side_y=0, **kw))
    full.init_fields(*fl)
    quarter = olb.create(inputs.RunParams(nx=M, ny=M, side_x=3, side_y=2, **kw))
    quarter.init_fields(*[v[:M, M:] for v in fl])
    assert full.step(20) == 0 and quarter.step(20) == 0
    a, b = quarter.get_populations(), full.get_populations()[:, :M, M:]
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_fp32_specular_close_to_fp64(olb):
    p, fl = setup(45, 19, 3, 2)
    a = olb.create(p, olb.FP64)
    b = olb.create(p, olb.FP32_KAHAN)
    a.init_fields(*fl)
    b.init_fields(*fl)
    assert a.step(10) == 0 and b.step(10) == 0
    r = moments_rel(b.moments(), a.moments())
    assert r["n"] < 1e-5 and r["T"] < 1e-5


def test_batch_with_specular_runs_equals_single_runs(olb):
    """A batch mixing every side kind advances each run exactly as a single
    context does (FP64, bit for bit)."""
    runs, fields = [], []
    for k, sides in enumerate(CONFIGS + [(1, 0), (0, 0)]):
        p, fl = setup(24 + 5 * k, 11 + 3 * k, *sides, seed=20 + k)
        runs.append(p)
        fields.append(fl)
    b = olb.Batch(runs)
    for r, fl in enumerate(fields):
        b.init_fields(r, *fl)
    assert b.step(3) == 0
    for r, (p, fl) in enumerate(zip(runs, fields)):
        c = olb.create(p)
        c.init_fields(*fl)
        assert c.step(3) == 0
        assert np.array_equal(b.get_populations(r), c.get_populations()), r


def test_invalid_specular_parameters_rejected(olb):
    for nx, ny, sx, sy in [(2, 5, 2, 0), (5, 2, 0, 2), (6, 6, 4, 0), (6, 6, 0, 1), (2, 4, 3, 0)]:
        p = inputs.RunParams(nx=nx, ny=ny, ds=0.1, dt=1e-3, tau=0.01, side_x=sx, side_y=sy)
        with pytest.raises(olb.OlbError):
            olb.create(p)
