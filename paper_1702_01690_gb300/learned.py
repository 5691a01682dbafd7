"""Training data and training of the learned WENO-5 weights.

The network (see olb_mlp_* in include/olb.h) replaces the Jiang-Shu weights
of Eq. weno5_omega.  Its training data come from this solver:

* fine-grid fields: populations of periodic runs (Laplace drops, waves,
  band-limited noise) advanced a few steps by the library's FP64 path;
* coarse stencils: every `ratio`-th node of a grid line, i.e. the five
  values the coarse scheme (spacing h = ratio ds) sees at an interface, in
  both upwind orientations;
* targets: the value a finite-difference WENO flux should take at the
  interface, h(x_{i+1/2}) of the function h whose cell averages (width h) are
  the point values f: h = f - h^2/24 f'' + 7 h^4/5760 f'''' + O(h^6) (the
  inverse of the cell-average operator), with f'' and f'''' from central
  differences of orders 6 and 4 on the fine line at the interface, which is a
  fine node when ratio is even.

Only stencils on which the network acts are kept: no vanishing smoothness
indicator (Table tab:weno applies there) and min sigma_q < 0.9 max sigma_q
(on smooth data sigma_min / sigma_max = 1 - O(h), so as the grid is refined
every smooth stencil passes to the Jiang-Shu weights, which approach the
ideal weights and keep 5th order).  Inputs are
normalised as x = (v - mean)/(max - min) (the network's input); the
candidate offsets G_q (Eq. weno5_flux minus the centre value) and the target
offset are divided by the same range.  Training runs on the GPU through
olb_mlp_train.
"""
from __future__ import annotations

import os

import numpy as np

from . import inputs


GUARD = 0.9


def _sigmas(V):
    V = np.asarray(V, dtype=np.float64)
    d = np.diff(V, axis=1)
    a1, b1 = d[:, 1] - d[:, 0], 3 * d[:, 1] - d[:, 0]
    a2, b2 = d[:, 2] - d[:, 1], d[:, 1] + d[:, 2]
    a3, b3 = d[:, 3] - d[:, 2], d[:, 3] - 3 * d[:, 2]
    return np.stack([13 * a1 ** 2 + 3 * b1 ** 2, 13 * a2 ** 2 + 3 * b2 ** 2, 13 * a3 ** 2 + 3 * b3 ** 2], axis=1)


def network_acts(V):
    """Rows of stencils V on which the network's weights are used."""
    S = _sigmas(V)
    return (~_js_sigma_zero(V)) & (S.min(axis=1) < GUARD * S.max(axis=1))


def _js_sigma_zero(V):
    """Rows of stencils V [S][5] with a vanishing smoothness indicator."""
    d = np.diff(V, axis=1)
    a1, b1 = d[:, 1] - d[:, 0], 3 * d[:, 1] - d[:, 0]
    a2, b2 = d[:, 2] - d[:, 1], d[:, 1] + d[:, 2]
    a3, b3 = d[:, 3] - d[:, 2], d[:, 3] - 3 * d[:, 2]
    return ((a1 == 0) & (b1 == 0)) | ((a2 == 0) & (b2 == 0)) | ((a3 == 0) & (b3 == 0))


def candidate_offsets(V):
    """G_q = F^q - v2 (Eq. weno5_flux) of upwind-ordered stencils V [S][5]."""
    v0, v1, v2, v3, v4 = np.asarray(V, dtype=np.float64).T
    return np.stack([(2 * v0 - 7 * v1 + 5 * v2) / 6, (-v1 - v2 + 2 * v3) / 6, (-4 * v2 + 5 * v3 - v4) / 6], axis=1)


def line_samples(line, ratio: int = 4):
    """Stencils, targets and the line's magnitude max |f| from one periodic
    fine line (ratio even)."""
    f = np.asarray(line, dtype=np.float64)
    L = f.size
    h = float(ratio)  # in fine-node units; targets are scale-free below
    # derivatives at every fine node (periodic), fine spacing 1
    s = lambda k: np.roll(f, -k)
    d2 = (s(3) + s(-3)) / 90 - 3 * (s(2) + s(-2)) / 20 + 1.5 * (s(1) + s(-1)) - 49 / 18 * f
    d4 = (-(s(3) + s(-3)) + 12 * (s(2) + s(-2)) - 39 * (s(1) + s(-1)) + 56 * f) / 6
    target = f - h * h / 24 * d2 + 7 * h ** 4 / 5760 * d4
    Vs, Ts = [], []
    for o in range(ratio):
        idx = (o + ratio * np.arange(L // ratio)) % L
        c = f[idx]
        n = c.size
        if n < 6:
            continue
        i = np.arange(n)
        face = (idx + ratio // 2) % L                    # fine node at x_{i+1/2}
        # p > 0: c_{i-2} .. c_{i+2};  p < 0: c_{i+3} .. c_{i-1}
        pos = np.stack([c[(i + k) % n] for k in (-2, -1, 0, 1, 2)], axis=1)
        neg = np.stack([c[(i + k) % n] for k in (3, 2, 1, 0, -1)], axis=1)
        Vs += [pos, neg]
        Ts += [target[face], target[face]]
    V, T = np.concatenate(Vs), np.concatenate(Ts)
    return V, T, np.full(len(T), np.abs(f).max())


def normalised_samples(V, t, s):
    """x, Gn, tn (float32) for stencils V and targets t, keeping only the
    stencils the network acts on; also returns the kept (V, t, r), r the
    stencil ranges (s, the line magnitudes, only filters empty lines)."""
    V = np.asarray(V, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    r = V.max(axis=1) - V.min(axis=1)
    keep = network_acts(V) & (r > 1e-13 * np.maximum(np.abs(V).max(axis=1), 1e-300)) & (s > 0)
    V, t, r, s = V[keep], t[keep], r[keep], s[keep]
    x = (V - V.mean(axis=1, keepdims=True)) / r[:, None]
    Gn = candidate_offsets(V) / r[:, None]
    tn = (t - V[:, 2]) / r
    return (x.astype(np.float32), Gn.astype(np.float32), tn.astype(np.float32)), (V, t, r)


def default_sources(scale: int = 1):
    """Periodic fine-grid runs used for training (steps to advance first)."""
    out = []
    n = 512 * scale
    for R in (0.1, 0.2, 0.3):
        p, f = inputs.laplace(n, R=R, steps=4)
        out.append((p, f, 4))
    ds = 1.0 / (256 * scale)
    p = inputs.RunParams(nx=256 * scale, ny=256 * scale, ds=ds, dt=inputs.stable_dt(ds), tau=0.01)
    for amp in (0.05, 0.2):
        out.append((p, inputs.shear_wave(p.nx, p.ny, ds, 1.0, 0.9, amp), 4))
        out.append((p, inputs.longitudinal_wave(p.nx, p.ny, ds, 1.0, 0.9, amp), 4))
    # waves resolved by 16 and 32 coarse nodes per wavelength (the coarse,
    # smooth regime of the 64 x 4 shear-decay run and coarser grids)
    for m in (2 * scale, 4 * scale):
        out.append((p, inputs.shear_wave(p.nx, p.ny, ds, 1.0, 0.8, 0.01, m=m), 4))
        out.append((p, inputs.longitudinal_wave(p.nx, p.ny, ds, 1.0, 1.1, 0.01, m=m), 4))
    ds = 1.0 / (512 * scale)
    p = inputs.RunParams(nx=512 * scale, ny=64, ds=ds, dt=inputs.stable_dt(ds, n_max=1.1), tau=0.005)
    n0 = 1.0 + 0.05 * inputs.band_limited_noise(p.nx, p.ny, inputs.SEED_BASE + 7, 8)
    z = np.zeros_like(n0)
    out.append((p, (n0, z, z.copy(), np.ones_like(n0)), 4))
    return out


def harvest(sources=None, ratio: int = 4, row_stride: int = 16, velocities=None):
    """Raw stencils V [S][5], targets t [S] and line magnitudes s [S] from
    solver runs (FP64 path)."""
    from . import olb
    if sources is None:
        sources = default_sources()
    moving = velocities if velocities is not None else [k for k in range(25) if k // 5 != 2]
    Vs, Ts, Ss = [], [], []
    for p, fields, steps in sources:
        ctx = olb.create(p)
        ctx.init_fields(*fields)
        ctx.step(steps)
        f = ctx.get_populations()
        ctx.close()
        for k in moving:
            for j in range(0, p.ny, row_stride):  # x lines (periodic runs only)
                V, t, s = line_samples(f[k, j, :], ratio)
                Vs.append(V)
                Ts.append(t)
                Ss.append(s)
    return np.concatenate(Vs), np.concatenate(Ts), np.concatenate(Ss)


def train(x, Gn, tn, epochs: int = 40, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Glorot-initialised network trained on the GPU; returns (theta as a
    numpy float32 array, loss history)."""
    import torch
    from . import olb
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(tn))
    x, Gn, tn = x[perm], Gn[perm], tn[perm]
    sizes = [(32, 5), (32,), (32, 32), (32,), (3, 32), (3,)]
    parts = []
    for shp in sizes:
        if len(shp) == 2:
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            parts.append(rng.uniform(-lim, lim, shp).ravel())
        else:
            parts.append(np.zeros(shp))
    theta = torch.tensor(np.concatenate(parts), dtype=torch.float32, device="cuda")
    hist = olb.mlp_train(theta, torch.from_numpy(x).cuda(), torch.from_numpy(Gn).cuda(),
                         torch.from_numpy(tn).cuda(), epochs, batch, lr)
    return theta.cpu().numpy(), hist


THETA_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weno_mlp_theta.txt")


def save_theta(theta, path: str = THETA_FILE) -> None:
    """Write the 1347 network parameters as text (9 significant digits, exact
    for float32)."""
    th = np.asarray(theta, dtype=np.float32).reshape(-1)
    assert th.size == 1347
    np.savetxt(path, th, fmt="%.9e", header="5-32-32-3 WENO-5 weight network, parameters W1 b1 W2 b2 W3 b3")


def load_theta(path: str = THETA_FILE) -> np.ndarray:
    """The parameters written by save_theta (float32)."""
    th = np.loadtxt(path, dtype=np.float64).astype(np.float32)
    assert th.size == 1347
    return th


def train_default(epochs: int = 30, seed: int = 0):
    """Harvest the default training runs and train on all their stencils
    (GPU); returns (theta, loss history, number of samples)."""
    V, t, s = harvest(default_sources(), ratio=4, row_stride=16)
    (x, Gn, tn), _ = normalised_samples(V, t, s)
    theta, hist = train(x, Gn, tn, epochs=epochs, batch=4096, lr=2e-3, seed=seed)
    return theta, hist, len(tn)


if __name__ == "__main__":
    # python -m paper_1702_01690_gb300.learned [path]: train the shipped network
    import sys
    theta, hist, n = train_default()
    save_theta(theta, sys.argv[1] if len(sys.argv) > 1 else THETA_FILE)
    print(f"trained on {n} stencils; loss per epoch {hist.tolist()}")
