"""olb_step_static: stepping a small grid without any device allocation.

Callers that must not call cudaMalloc / cudaFree while they step (those
calls synchronise the device; some hosts own all device memory) use this
entry point: the caller passes the populations, the library keeps its two
intermediate RK-3 buffers in a fixed device array.  The test drives it
through the C ABI and compares it with olb_step on the same inputs, over two
calls in a row and on grids of other shapes (a ragged 45 x 19 grid with
walls, whose unpadded rows differ from the library's padded layout, against
the oracle as well, and a grid of exactly the largest accepted size), within
the FP64 tolerance of the other parity tests.  It sits in a file of its own that
pytest collects last, and passes alone in a fresh process as well as after
the other tests."""
import ctypes

import numpy as np
import pytest

from helpers import field_rel, make_oracle
from paper_1702_01690_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


@pytest.fixture(scope="module")
def olb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01690_gb300 import build
    build.build()
    from paper_1702_01690_gb300 import olb as mod
    return mod


def static_steps(olb, params, dev_f, nsteps):
    import torch
    stream = torch.cuda.current_stream()
    return olb.library().olb_step_static(ctypes.byref(params), ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.c_void_p(dev_f.data_ptr()), int(nsteps))


def test_static_step_matches_olb_step(olb):
    import torch
    # planar workload at full size (8192 nodes), then a periodic grid of another shape
    for p, fields in (inputs.planar_walls(), inputs.shear_64x4()):
        params = olb.params_from(p)
        ctx = olb.create(p)
        ctx.init_fields(*fields)
        dev = torch.from_numpy(ctx.get_populations()).cuda().contiguous()
        for _ in range(2):  # two calls in a row share the static scratch
            ctx.step(3)
            assert static_steps(olb, params, dev, 3) == olb.OK
            ref = ctx.get_populations()
            got = dev.cpu().numpy()
            assert field_rel(got, ref) < FP64_TOL
        ctx.close()


def test_static_step_ragged_grid_matches_oracle(olb):
    """45 x 19 with diffuse walls: the caller's [25][19][45] array has rows
    of 45 values (the library's own buffers pad rows to 64)."""
    import torch
    p = inputs.RunParams(nx=45, ny=19, ds=1.0 / 45, dt=0.2 / 45 / inputs.P_MAX, tau=0.01,
                         Tw=(0.85, 0.95), uw=(0.01, -0.02), side_x=1)
    rng = np.random.default_rng(45)
    n = 1.0 + 0.05 * rng.uniform(-1, 1, (19, 45))
    ux, uy = 0.01 * rng.uniform(-1, 1, (2, 19, 45))
    T = np.full((19, 45), 0.95)
    o = make_oracle(p, (n, ux, uy, T))
    dev = torch.from_numpy(o.get_populations()).cuda().contiguous()
    for _ in range(2):
        o.step(4)
        assert static_steps(olb, olb.params_from(p), dev, 4) == olb.OK
        assert field_rel(dev.cpu().numpy(), o.get_populations()) < FP64_TOL


def test_static_step_at_the_size_limit(olb):
    """Exactly OLB_STATIC_MAX_NODES nodes (128 x 128 periodic): f^(2) then
    ends where the status word starts."""
    import torch
    N = 128
    assert N * N == olb.STATIC_MAX_NODES
    ds = 1.0 / N
    p = inputs.RunParams(nx=N, ny=N, ds=ds, dt=inputs.stable_dt(ds), tau=0.01)
    fields = inputs.shear_wave(N, N, ds, 1.0, 1.0, 1e-2)
    ctx = olb.create(p)
    ctx.init_fields(*fields)
    dev = torch.from_numpy(ctx.get_populations()).cuda().contiguous()
    ctx.step(3)
    assert static_steps(olb, olb.params_from(p), dev, 3) == olb.OK
    assert field_rel(dev.cpu().numpy(), ctx.get_populations()) < FP64_TOL
    ctx.close()


def test_static_step_rejects_large_grid(olb):
    import torch
    p = inputs.RunParams(nx=129, ny=128, ds=1 / 129, dt=1e-4, tau=0.01)
    assert p.nx * p.ny > olb.STATIC_MAX_NODES
    dev = torch.zeros((25, p.ny, p.nx), dtype=torch.float64, device="cuda")
    assert static_steps(olb, olb.params_from(p), dev, 1) == olb.ERR_ARG
    fp32 = olb.params_from(inputs.shear_64x4()[0], olb.FP32_KAHAN)
    assert static_steps(olb, fp32, dev, 1) == olb.ERR_ARG
    # specular sides and learned weights are not accepted either
    q = inputs.RunParams(nx=32, ny=32, ds=1 / 32, dt=1e-4, tau=0.01, side_y=2)
    assert static_steps(olb, olb.params_from(q), dev, 1) == olb.ERR_ARG
    q = inputs.RunParams(nx=32, ny=32, ds=1 / 32, dt=1e-4, tau=0.01)
    assert static_steps(olb, olb.params_from(q, olb.FP64, olb.WENO_LEARNED), dev, 1) == olb.ERR_ARG
