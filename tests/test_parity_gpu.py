"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 contract: n, u, T within 1e-11 of the oracle relative to each field's
magnitude after 200 steps of the shear-wave workload, and on the coarse and
ragged grids; populations within 1e-12 after single steps.  On fine grids
with smooth fields the force stencils are ill-conditioned (they cancel to
O(ds^3) of their terms), so there each field must lie within
max(1e-11 x magnitude, 10 x the rounding envelope): the spread of two oracle
runs whose states differ by a few ulp per step (helpers.rounding_envelope).
FP32 (compensated hi + lo storage): n, u and T within 1e-5 of the FP64
oracle, relative to each field's magnitude, on the planar wall workload at
its full size (1024 x 8, 200 steps) and on windows of the Laplace-drop
workload at its full size (2048^2, 10 steps)."""
import math

import numpy as np
import pytest

from helpers import check_against_envelope, field_rel, make_oracle, moments_rel, rounding_envelope
from paper_1702_01690_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def olb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_01690_gb300 import build
    build.build()
    from paper_1702_01690_gb300 import olb as mod
    return mod


def run_pair(olb, p, fields, steps, precision=0):
    ctx = olb.create(p, precision)
    ctx.init_fields(*fields)
    o = make_oracle(p, fields)
    if steps:
        assert ctx.step(steps) == 0
        o.step(steps)
    return ctx, o


def noisy(p, seed=5, amp=0.01, T0=1.0, uamp=0.0):
    n, ux, uy, T = inputs.noisy_rest(p.nx, p.ny, seed, 1.0, amp, T0)
    if uamp:
        rng = np.random.default_rng(seed + 1)
        ux = uamp * rng.uniform(-1, 1, n.shape)
        uy = uamp * rng.uniform(-1, 1, n.shape)
    return n, ux, uy, T


# ------------------------------------------------------------------ basics

def test_init_is_equilibrium(olb):
    p, fl = inputs.shear_64x4()
    ctx, o = run_pair(olb, p, fl, 0)
    assert field_rel(ctx.get_populations(), o.get_populations()) < 1e-14
    m = ctx.moments()
    for a, b in zip(m, fl):
        assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("side_x", [0, 1])
def test_one_step_populations(olb, side_x):
    p, _ = inputs.planar_walls(nx=40, ny=8)
    p.side_x = side_x
    ctx, o = run_pair(olb, p, noisy(p, uamp=0.02), 1)
    assert field_rel(ctx.get_populations(), o.get_populations()) < 1e-12


def test_shear_wave_200_steps_fp64(olb):
    """Shear-wave workload (64 x 4, 200 RK-3 steps): 1e-11 on n, u, T."""
    p, fl = inputs.shear_64x4()
    ctx, o = run_pair(olb, p, fl, p.steps)
    err = moments_rel(ctx.moments(), o.moments())
    assert max(err.values()) < FP64_TOL, err


@pytest.mark.parametrize("nx,ny,side_x", [(37, 11, 0), (45, 3, 1), (3, 1, 1), (1, 5, 0), (70, 9, 1), (33, 17, 0)])
def test_ragged_and_tiny_grids(olb, nx, ny, side_x):
    """Grids that leave ragged tiles, fewer rows than the stencil, and the
    smallest wall domain (nx = 3)."""
    p = inputs.RunParams(nx=nx, ny=ny, ds=1.0 / max(nx, 8), dt=0.2 / max(nx, 8) / inputs.P_MAX,
                         tau=0.01, Tw=(0.85, 0.95), uw=(0.01, -0.02), side_x=side_x)
    ctx, o = run_pair(olb, p, noisy(p, seed=nx * 31 + ny, amp=0.05, uamp=0.01), 10)
    err = moments_rel(ctx.moments(), o.moments())
    assert max(err.values()) < FP64_TOL, err
    assert field_rel(ctx.get_populations(), o.get_populations()) < FP64_TOL


def test_planar_walls_full_grid(olb):
    """Planar-interface workload at its full size (1024 x 8, diffuse walls,
    the launch configuration of the wall workloads) for 200 steps: the
    populations and n, T within 1e-11 of the oracle relative to their
    magnitude; u (which the force creates from rest, a small difference of
    O(1) populations) within max(1e-11 x |u|max, 10 x the rounding envelope)."""
    p, fl = inputs.planar_walls()
    ctx = olb.create(p)
    ctx.init_fields(*fl)
    assert ctx.step(200) == 0
    env, o = rounding_envelope(p, fl, 200)
    assert field_rel(ctx.get_populations(), o.get_populations()) < FP64_TOL
    m, ref = ctx.moments(), o.moments()
    assert field_rel(m[0], ref[0]) < FP64_TOL
    assert field_rel(m[3], ref[3]) < FP64_TOL
    us = max(np.max(np.abs(ref[1])), np.max(np.abs(ref[2])))
    for k in (1, 2):
        allowed = max(FP64_TOL * us, 10.0 * float(np.max(env[k])))
        assert np.max(np.abs(m[k] - ref[k])) < allowed, (k, np.max(np.abs(m[k] - ref[k])), allowed)


@pytest.mark.parametrize("V", [0.5, 2.0])
def test_background_velocity_matches_oracle(olb, V):
    """Shear wave carried at a background velocity V along x (the Galilean
    runs of Sec. 6.1: T0 = 0.8, tau = 5e-4, dt = 2e-4) on a 32 x 4 periodic
    grid, 100 steps: n, u, T within 1e-11 of the oracle (u relative to the
    largest |u|, here V)."""
    N = 32
    ds = 1.0 / N
    p = inputs.RunParams(nx=N, ny=4, ds=ds, dt=2e-4, tau=5e-4, a=0.0, b=0.0)
    fl = inputs.shear_wave(N, 4, ds, 1.0, 0.8, 1e-3, V=V)
    ctx, o = run_pair(olb, p, fl, 100)
    err = moments_rel(ctx.moments(), o.moments())
    assert max(err.values()) < FP64_TOL, err
    assert field_rel(ctx.get_populations(), o.get_populations()) < FP64_TOL


def test_graph_replay_matches_single_steps(olb):
    """16-step graph + 1-step graph replay = 17 single-step calls, bit for bit."""
    p, _ = inputs.planar_walls(nx=48, ny=8)
    fl = noisy(p)
    a = olb.create(p)
    a.init_fields(*fl)
    a.step(17)
    b = olb.create(p)
    b.init_fields(*fl)
    for _ in range(17):
        b.step(1)
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_set_get_populations_roundtrip_and_resume(olb):
    """Checkpoint / resume: stepping 5 + 5 with a host round trip in between
    equals 10 continuous steps bit for bit."""
    p, _ = inputs.planar_walls(nx=40, ny=6)
    fl = noisy(p)
    a = olb.create(p)
    a.init_fields(*fl)
    a.step(10)
    b = olb.create(p)
    b.init_fields(*fl)
    b.step(5)
    snap = b.get_populations()
    c = olb.create(p)
    c.set_populations(snap)
    c.step(5)
    assert np.array_equal(a.get_populations(), c.get_populations())


def test_device_entry_points(olb):
    import torch
    p, fl = inputs.shear_64x4()
    ctx = olb.create(p)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fl]
    ctx.init_fields(*dev)
    ctx.step_async(3)
    assert ctx.status() == 0
    md = [t.cpu().numpy() for t in ctx.moments_device()]
    torch.cuda.synchronize()
    mh = ctx.moments()
    for a, b in zip(md, mh):
        assert np.array_equal(a, b)
    o = make_oracle(p, fl)
    o.step(3)
    assert max(moments_rel(mh, o.moments()).values()) < FP64_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_host_buffers_match_pageable(olb, precision):
    """Pinned host arrays (read and written by the kernels directly) give the
    same state and moments, bit for bit, as pageable ones (staging copies);
    NULL skips a moment; invalid pinned input is still rejected."""
    import torch
    p, fl = inputs.shear_64x4()
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fl]
    a = olb.create(p, precision)
    b = olb.create(p, precision)
    a.init_fields(*fl)
    olb._check(olb.library().olb_init_fields(b.handle, *[olb._VP(t.data_ptr()) for t in pinned]), "init")
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.step(5)
    b.step(5)
    out = [torch.zeros((p.ny, p.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    ptrs = [olb._VP(t.data_ptr()) for t in out]
    ptrs[2] = None
    olb._check(olb.library().olb_moments(b.handle, *ptrs), "moments")
    ma = a.moments()
    for k in (0, 1, 3):
        assert np.array_equal(out[k].numpy(), ma[k])
    assert not out[2].numpy().any()
    bad = [t.clone().pin_memory() for t in pinned]
    bad[3][0, 0] = -1.0
    rc = olb.library().olb_init_fields(b.handle, *[olb._VP(t.data_ptr()) for t in bad])
    assert rc == olb.ERR_ARG


def test_diverged_state_reported(olb):
    """A state with negative density is reported as OLB_ERR_DIVERGED by the
    status word, never as a device fault."""
    p, fl = inputs.shear_64x4()
    ctx = olb.create(p)
    ctx.init_fields(*fl)
    ctx.set_populations(-np.abs(ctx.get_populations()))
    rc = olb.library().olb_step(ctx.handle, 1)
    assert rc == olb.ERR_DIVERGED
    ctx.init_fields(*fl)  # init clears the status
    assert ctx.step(1) == 0


def test_init_fields_rejects_invalid_values(olb):
    p, fl = inputs.shear_64x4()
    ctx = olb.create(p)
    n, ux, uy, T = [a.copy() for a in fl]
    n[0, 0] = -1.0
    with pytest.raises(olb.OlbError):
        ctx.init_fields(n, ux, uy, T)
    n[0, 0] = 3.5  # b n >= 1
    with pytest.raises(olb.OlbError):
        ctx.init_fields(n, ux, uy, T)
    with pytest.raises(olb.OlbError):
        ctx.step(1)  # not initialised


def test_init_fields_rejects_invalid_values_on_large_grids(olb):
    """Grids above 2^19 nodes are checked by several host threads: one bad
    value in any part of any field is still rejected, pinned host arrays
    included, and a valid state is accepted afterwards."""
    import torch
    N = 1024
    ds = 1.0 / N
    p = inputs.RunParams(nx=N, ny=N, ds=ds, dt=inputs.stable_dt(ds), tau=0.01)
    fl = inputs.shear_wave(N, N, ds, 1.0, 1.0, 1e-3)
    ctx = olb.create(p)
    for which, (j, i), bad in ((0, (0, 0), -1.0), (3, (N - 1, N - 1), 0.0), (1, (N // 2, 7), np.nan),
                               (2, (700, 1000), np.inf), (0, (300, 300), 3.5)):
        arrs = [a.copy() for a in fl]
        arrs[which][j, i] = bad
        with pytest.raises(olb.OlbError):
            ctx.init_fields(*arrs)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fl]
    pinned[3][N - 1, 0] = -0.5
    with pytest.raises(olb.OlbError):
        ctx.init_fields(*[t.numpy() for t in pinned])
    pinned[3][N - 1, 0] = 1.0
    ctx.init_fields(*[t.numpy() for t in pinned])
    assert ctx.step(1) == 0
    ctx.close()


# ------------------------------------------------------------------ full-size samples

def crop_window(fields, x0, y0, wx, wy, nx, ny, periodic_x):
    """Sub-window [x0, x0+wx) x [y0, y0+wy) of (ny, nx) fields with y (and x
    when periodic) wrapped."""
    ys = np.arange(y0, y0 + wy) % ny
    xs = np.arange(x0, x0 + wx)
    if periodic_x:
        xs = xs % nx
    return tuple(np.ascontiguousarray(a[np.ix_(ys, xs)]) for a in fields)


def window_check(olb, p, fields, windows, margin=10, steps=1):
    """One GPU run at full size; the oracle on windows around sample points.
    A node depends on nodes at most 3 away per stage (WENO stencil and the
    49-point stencils of pointwise moments), 9 per RK-3 step, so the window
    interior more than 9*steps from a cut edge is exact.  The populations and
    n, T must agree within 1e-11 of their magnitude over the whole grid; u,
    which one step only just creates and which is a small difference of O(1)
    populations, within max(1e-11 x |u|max, 10 x the largest spread of the
    rounding envelope over the window interior).  Returns the worst error / allowed ratio and per-window,
    per-field details."""
    ctx = olb.create(p)
    ctx.init_fields(*fields)
    assert ctx.step(steps) == 0
    m_gpu = ctx.moments()
    f_gpu = ctx.get_populations()
    fscale = np.max(np.abs(f_gpu))
    us = max(np.max(np.abs(m_gpu[1])), np.max(np.abs(m_gpu[2])))
    scale = [np.max(np.abs(m_gpu[0])), us, us, np.max(np.abs(m_gpu[3]))]
    worst = 0.0
    details = []
    for (x0, y0, wx, wy, at_wall) in windows:
        wp = inputs.RunParams(**{**p.as_dict(), "nx": wx, "ny": wy})
        if not at_wall:
            wp.side_x = 0
        sub = crop_window(fields, x0, y0, wx, wy, p.nx, p.ny, p.side_x == 0)
        env, o = rounding_envelope(wp, sub, steps)
        mo = o.moments()
        fo = o.get_populations()
        inner_y = slice(margin * steps, wy - margin * steps)
        if at_wall == "left":
            inner_x = slice(0, wx - margin * steps)
        elif at_wall == "right":
            inner_x = slice(margin * steps, wx)
        else:
            inner_x = slice(margin * steps, wx - margin * steps)
        ys = np.arange(y0, y0 + wy) % p.ny
        xs = np.arange(x0, x0 + wx) % p.nx
        fg = f_gpu[:, ys][:, :, xs][:, inner_y, inner_x]
        ratio_f = float(np.max(np.abs(fg - fo[:, inner_y, inner_x])) / (FP64_TOL * fscale))
        details.append(dict(window=(x0, y0), field="f", ratio=ratio_f, gpu=0.0, oracle=0.0, env=0.0,
                            scale=float(fscale), at=(0, 0)))
        worst = max(worst, ratio_f)
        for k in range(4):
            g = m_gpu[k][np.ix_(ys, xs)][inner_y, inner_x]
            r = mo[k][inner_y, inner_x]
            e = env[k][inner_y, inner_x]
            allowed = np.full(g.shape, FP64_TOL * scale[k])
            if k in (1, 2):
                allowed = np.maximum(allowed, 10.0 * float(np.max(e)))
            ratio = np.abs(g - r) / allowed
            q = np.unravel_index(np.argmax(ratio), ratio.shape)
            details.append(dict(window=(x0, y0), field="n ux uy T".split()[k], ratio=float(ratio[q]),
                                gpu=float(g[q]), oracle=float(r[q]), env=float(e[q]), scale=float(scale[k]),
                                at=(int(q[0]), int(q[1]))))
            worst = max(worst, float(ratio[q]))
    return worst, details


def fmt_detail(d):
    return (f"window {d['window']} {d['field']} at {d['at']}: ratio {d['ratio']:.3g} gpu {d['gpu']:.17g} "
            f"oracle {d['oracle']:.17g} envelope {d['env']:.3g} scale {d['scale']:.3g}")


def test_laplace_2048_sampled_windows(olb):
    """Laplace-drop workload at full size (2048^2 periodic) after one step,
    sampled on oracle windows across the drop interface and in the bulk."""
    p, fl = inputs.laplace(2048, R=0.2, steps=1)
    wins = [(1024 - 20 + dx, 1024 + 410 - 20 + dy, 40, 40, None) for dx, dy in ((0, 0), (300, -100))]
    wins += [(2048 - 20, 2048 - 20, 40, 40, None)]  # wraps both axes
    worst, details = window_check(olb, p, fl, wins)
    assert worst < 1.0, "; ".join(fmt_detail(d) for d in details if d["ratio"] > 0.3)


def test_phase_separation_4096_sampled_windows(olb):
    """Cold-plate workload at full size (4096^2, diffuse walls) after one step,
    sampled on oracle windows at both walls and in the bulk."""
    p, fl = inputs.phase_separation(4096, steps=1)
    wins = [(0, 100, 40, 40, "left"), (4096 - 40, 3000, 40, 40, "right"), (2000, 4096 - 20, 40, 40, None)]
    worst, details = window_check(olb, p, fl, wins)
    assert worst < 1.0, "; ".join(fmt_detail(d) for d in details if d["ratio"] > 0.3)


# ------------------------------------------------------------------ FP32 (compensated storage)

def test_fp32_kahan_shear_wave(olb):
    """Shear-wave workload (64 x 4, 200 steps) in FP32: n, u, T against the
    FP64 oracle."""
    p, fl = inputs.shear_64x4()
    ctx, o = run_pair(olb, p, fl, p.steps, precision=olb.FP32_KAHAN)
    err = moments_rel(ctx.moments(), o.moments())
    print("fp32 shear vs oracle", err)
    assert max(err.values()) < FP32_TOL, err


def test_fp32_kahan_planar_walls(olb):
    """Planar wall workload at its full size (1024 x 8, 200 steps) in FP32:
    n, u, T within 1e-5 of the FP64 oracle."""
    p, fl = inputs.planar_walls()
    ctx, o = run_pair(olb, p, fl, 200, precision=olb.FP32_KAHAN)
    err = moments_rel(ctx.moments(), o.moments())
    print("fp32 planar vs oracle", err)
    assert max(err.values()) < FP32_TOL, err


def test_planar_workload_long_run_conserves_mass(olb):
    """Planar workload at full size for 2000 steps: stays valid (status OK),
    total mass constant to rounding (zero net wall flux, Eq. nw), and the
    liquid starts to form at the cold walls (density rises there)."""
    p, fl = inputs.planar_walls()
    ctx = olb.create(p)
    ctx.init_fields(*fl)
    m0 = ctx.moments()[0]
    assert ctx.step(2000) == 0
    m = ctx.moments()
    assert abs(m[0].sum() - m0.sum()) < 1e-12 * m0.sum()
    assert np.all(np.isfinite(m[3])) and m[3].min() > 0.85
    assert m[0][:, :8].mean() > m0[:, :8].mean()


@pytest.mark.parametrize("side_x", [0, 1])
def test_every_tile_shape_gives_identical_results(olb, side_x):
    """The stage kernel's shapes (tile size, velocity lanes) only change which
    thread computes what: populations agree bit for bit."""
    p = inputs.RunParams(nx=45, ny=19, ds=1.0 / 45, dt=0.2 / 45 / inputs.P_MAX, tau=0.01,
                         Tw=(0.85, 0.95), side_x=side_x)
    fl = noisy(p, seed=9, amp=0.05, uamp=0.01)
    ref = None
    for shape in ((8, 8, 4), (16, 8, 2), (16, 8, 1), (32, 8, 1), (8, 8, 8), (7, 8, 8), (8, 8, 5)):
        ctx = olb.create(p)
        ctx.set_tile(*shape)
        assert ctx.get_tile() == shape
        ctx.init_fields(*fl)
        ctx.step(4)
        f = ctx.get_populations()
        if ref is None:
            ref = f
            o = make_oracle(p, fl)
            o.step(4)
            assert field_rel(f, o.get_populations()) < FP64_TOL
        else:
            assert np.array_equal(f, ref), shape
    with pytest.raises(olb.OlbError):
        ctx.set_tile(8, 8, 1)
    ctx.set_tile(32, 16, 1)
    ctx.init_fields(*fl)
    ctx.step(4)
    assert np.array_equal(ctx.get_populations(), ref)


@pytest.mark.parametrize("side_x", [0, 1])
def test_every_tile_shape_gives_identical_results_fp32(olb, side_x):
    """FP32: the small tiles compute their faces in strips that carry
    differences and squares from face to face, the large tiles one face at a
    time; the arithmetic is the same, so every shape agrees bit for bit."""
    p = inputs.RunParams(nx=45, ny=19, ds=1.0 / 45, dt=0.2 / 45 / inputs.P_MAX, tau=0.01,
                         Tw=(0.85, 0.95), side_x=side_x)
    fl = noisy(p, seed=9, amp=0.05, uamp=0.01)
    ref = None
    for shape in ((32, 16, 1), (8, 8, 4), (16, 8, 2), (16, 8, 1), (32, 8, 1), (8, 8, 8), (7, 8, 8), (8, 8, 5)):
        ctx = olb.create(p, olb.FP32_KAHAN)
        ctx.set_tile(*shape)
        ctx.init_fields(*fl)
        assert ctx.step(4) == 0
        f = ctx.get_populations()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref), shape


def test_fp32_kahan_laplace_2048_windows(olb):
    """Laplace-drop workload at its full size (2048^2 periodic) in FP32, 10
    steps, against the FP64 oracle on windows across the drop interface and
    in the bulk: n, u, T within 1e-5 of each field's largest value over the
    grid (u: the largest |u_x|, |u_y|; far from the drop u is ~0).  (On this
    grid the capillary stencil cancels ~10^3-fold; the FP32 path sums it in
    double-float arithmetic.)"""
    steps = 10
    p, fl = inputs.laplace(2048, R=0.2, steps=steps)
    ctx = olb.create(p, olb.FP32_KAHAN)
    ctx.init_fields(*fl)
    assert ctx.step(steps) == 0
    m = ctx.moments()
    scale = {"n": np.max(np.abs(m[0])), "u": max(np.max(np.abs(m[1])), np.max(np.abs(m[2]))),
             "T": np.max(np.abs(m[3]))}
    margin = 10 * steps
    w = 40 + 2 * margin
    worst = {"n": 0.0, "u": 0.0, "T": 0.0}
    for x0, y0 in ((1024 - w // 2, 1024 + 410 - w // 2), (1024 + 300 - w // 2, 1024 + 310 - w // 2), (2048 - 60, 2048 - 60)):
        wp = inputs.RunParams(**{**p.as_dict(), "nx": w, "ny": w})
        sub = crop_window(fl, x0, y0, w, w, p.nx, p.ny, True)
        o = make_oracle(wp, sub)
        o.step(steps)
        ref = [a[margin:-margin, margin:-margin] for a in o.moments()]
        ys = np.arange(y0, y0 + w) % p.ny
        xs = np.arange(x0, x0 + w) % p.nx
        got = [a[np.ix_(ys, xs)][margin:-margin, margin:-margin] for a in m]
        e = {"n": np.max(np.abs(got[0] - ref[0])), "u": max(np.max(np.abs(got[1] - ref[1])), np.max(np.abs(got[2] - ref[2]))),
             "T": np.max(np.abs(got[3] - ref[3]))}
        worst = {k: max(worst[k], float(e[k] / scale[k])) for k in worst}
    print("fp32 laplace 2048 windows vs oracle", worst)
    assert max(worst.values()) < FP32_TOL, worst


# ------------------------------------------------------------------ global sums

def host_totals(p, m):
    """Mass, momentum and particle energy of moments m = (n, ux, uy, T) summed
    on the host in FP64 (times ds^2): sum n, n u, n (T + |u|^2 / 2)."""
    n, ux, uy, T = m
    return np.array([n.sum(), (n * ux).sum(), (n * uy).sum(), (n * (T + 0.5 * (ux ** 2 + uy ** 2))).sum()]) * p.ds ** 2


@pytest.mark.parametrize("precision", [0, 1])
def test_totals_match_oracle_sums(olb, precision):
    """olb_totals (GPU reduction in FP64) against the oracle's state summed on
    the host after 10 steps of a noisy moving run between diffuse walls: mass
    and energy to 1e-12 (FP64) / 1e-6 (FP32, whose state differs from the
    oracle's at that level), momentum relative to sum n |u| ds^2; repeated calls
    agree bit for bit."""
    p = inputs.RunParams(nx=45, ny=19, ds=1.0 / 45, dt=0.2 / 45 / inputs.P_MAX, tau=0.01,
                         Tw=(0.85, 0.95), uw=(0.01, -0.02), side_x=1)
    fl = noisy(p, seed=11, amp=0.05, uamp=0.01)
    ctx, o = run_pair(olb, p, fl, 10, precision)
    got = ctx.totals()
    assert np.array_equal(got, ctx.totals())
    m = o.moments()
    ref = host_totals(p, m)
    tol = 1e-12 if precision == 0 else 1e-6
    assert abs(got[0] - ref[0]) < tol * ref[0]
    assert abs(got[3] - ref[3]) < tol * ref[3]
    jscale = (m[0] * np.hypot(m[1], m[2])).sum() * p.ds ** 2
    assert np.max(np.abs(got[1:3] - ref[1:3])) < tol * jscale


@pytest.mark.parametrize("precision", [0, 1])
def test_step_totals_conserve_mass_between_walls(olb, precision):
    """olb_step_totals on the planar workload (256 x 8, diffuse walls): the
    records taken every 10 steps keep the mass to 1e-13 (FP64) / 1e-9 (FP32
    compensated) of itself (zero net wall flux, Eq. nw), the last record equals
    olb_totals afterwards, and the stepping equals olb_step bit for bit."""
    p, fl = inputs.planar_walls(nx=256, ny=8)
    a = olb.create(p, precision)
    a.init_fields(*fl)
    m0 = a.totals()[0]
    rec = a.step_totals(100, 10)
    assert rec.shape == (10, 4)
    assert np.array_equal(rec[-1], a.totals())
    tol = 1e-13 if precision == 0 else 1e-9
    assert np.max(np.abs(rec[:, 0] - m0)) < tol * m0, rec[:, 0] - m0
    b = olb.create(p, precision)
    b.init_fields(*fl)
    b.step(100)
    assert np.array_equal(a.get_populations(), b.get_populations())
