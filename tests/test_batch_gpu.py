"""Batched runs (one launch per stage over the tiles of many grids) against the
single-grid path and the oracle, and the autotuner."""
import numpy as np
import pytest

from helpers import field_rel, make_oracle
from paper_1702_01690_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def olb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01690_gb300 import build
    build.build()
    from paper_1702_01690_gb300 import olb as mod
    return mod


def small_batch():
    runs = []
    for nx, ny, side in ((40, 8, 1), (64, 4, 0), (33, 17, 0), (3, 1, 1), (70, 30, 1), (16, 16, 0)):
        ds = 1.0 / max(nx, 8)
        p = inputs.RunParams(nx=nx, ny=ny, ds=ds, dt=0.25 * ds / inputs.P_MAX, tau=0.01,
                             Tw=(0.8 + 0.01 * nx % 7, 0.9), uw=(0.0, 0.01), side_x=side)
        n, ux, uy, T = inputs.noisy_rest(nx, ny, 100 + nx, 1.0, 0.03, 0.95)
        rng = np.random.default_rng(nx)
        ux = 0.01 * rng.uniform(-1, 1, n.shape)
        runs.append((p, (n, ux, uy, T)))
    return runs


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_contexts(olb, precision):
    """Every run of a batch evolves as the same run in its own context (same
    stage code): bit for bit in FP64; in FP32 within FP32 rounding, since
    separately compiled kernels may contract FP32 expressions differently."""
    runs = small_batch()
    b = olb.Batch([p for p, _ in runs], precision)
    for r, (p, fl) in enumerate(runs):
        b.init_fields(r, *fl)
    assert b.step(5) == 0
    for r, (p, fl) in enumerate(runs):
        ctx = olb.create(p, precision)
        ctx.init_fields(*fl)
        ctx.step(5)
        if precision == 0:
            assert np.array_equal(b.get_populations(r), ctx.get_populations()), r
        else:
            assert field_rel(b.get_populations(r), ctx.get_populations()) < 1e-6, r
        ctx.close()
    rc, per = b.status()
    assert rc == 0 and not per.any()


@pytest.mark.parametrize("precision,shape", [(0, (8, 8, 4)), (0, (16, 8, 2)), (1, (8, 8, 8)), (1, (8, 8, 5)),
                                             (1, (32, 16, 1))])
def test_batch_tma_tiles_match_single_contexts(olb, precision, shape):
    """Runs large enough that most tiles lie inside their run (staged by one
    TMA copy from the run's own tensor map, the maps of the two runs side by
    side in device memory); walls on one run, periodic on the other."""
    runs = []
    for nx, ny, side in ((256, 256, 0), (200, 120, 1)):
        ds = 1.0 / nx
        p = inputs.RunParams(nx=nx, ny=ny, ds=ds, dt=0.25 * ds / inputs.P_MAX, tau=0.01,
                             Tw=(0.85, 0.9), uw=(0.0, 0.01), side_x=side)
        n, ux, uy, T = inputs.noisy_rest(nx, ny, 7 + nx, 1.0, 0.03, 0.95)
        runs.append((p, (n, 0.01 * np.sin(np.arange(nx) / 9.0)[None, :] + 0 * n, uy, T)))
    b = olb.Batch([p for p, _ in runs], precision)
    b.set_tile(*shape)
    for r, (p, fl) in enumerate(runs):
        b.init_fields(r, *fl)
    assert b.step(3) == 0
    for r, (p, fl) in enumerate(runs):
        ctx = olb.create(p, precision)
        ctx.set_tile(*shape)
        ctx.init_fields(*fl)
        ctx.step(3)
        if precision == 0:
            assert np.array_equal(b.get_populations(r), ctx.get_populations()), r
        else:
            assert field_rel(b.get_populations(r), ctx.get_populations()) < 1e-6, r
        ctx.close()
    rc, per = b.status()
    assert rc == 0 and not per.any()


def test_batch_matches_oracle(olb):
    runs = small_batch()
    b = olb.Batch([p for p, _ in runs])
    for r, (p, fl) in enumerate(runs):
        b.init_fields(r, *fl)
    b.step(3)
    for r in (0, 3, 4):
        p, fl = runs[r]
        o = make_oracle(p, fl)
        o.step(3)
        assert field_rel(b.get_populations(r), o.get_populations()) < 1e-11


def test_batch_autotune_keeps_state_and_results(olb):
    runs = small_batch()
    b = olb.Batch([p for p, _ in runs])
    for r, (p, fl) in enumerate(runs):
        b.init_fields(r, *fl)
    before = [b.get_populations(r) for r in range(b.count)]
    shape = b.autotune(2)
    assert shape == b.get_tile()
    for r in range(b.count):
        assert np.array_equal(b.get_populations(r), before[r])
    b.step(4)
    ref = olb.Batch([p for p, _ in runs])
    ref.set_tile(8, 8, 4)
    for r, (p, fl) in enumerate(runs):
        ref.init_fields(r, *fl)
    ref.step(4)
    for r in range(b.count):
        assert np.array_equal(b.get_populations(r), ref.get_populations(r))
    assert b.profile(2) > 0


def test_batch_sweep_workload_runs(olb):
    """The 64-run sweep (capped at 256^2 here) steps without divergence."""
    runs = inputs.batch_sweep(max_n=256)
    assert len(runs) == 64
    b = olb.Batch([p for p, _ in runs], olb.FP32_KAHAN)
    for r, (p, fl) in enumerate(runs):
        b.init_fields(r, *fl)
    assert b.step(20) == 0
