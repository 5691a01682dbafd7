"""Seeded synthetic initial conditions and run parameters.

This module is shared by the CUDA path, the tests and the benchmark.  It
holds no arithmetic of the method itself: it only builds initial fields
(n, u_x, u_y, T) on the node positions x = (i + 1/2) ds, y = (j + 1/2) ds and
the parameter sets of the workloads.  The paper uses no external dataset;
every workload is synthetic with the shapes and value distributions of its
experiments:

  shear wave      u_y = u0 sin(2 pi x), uniform n, T        (Sec. 6.1)
  planar walls    n = 1 + 0.01 noise, T = 1, diffuse walls   (Sec. 7 noise
                  at x = 0, 1                                recipe, Sec. 4 walls)
  Laplace drop    tanh drop of radius R, vapour outside      (Sec. 5)
  planar tanh     liquid slabs at the walls, Eq. tanh       (Sec. 4)
  Laplace bubble  gas bubble in the reduced (specular-sided) (Sec. 5)
                  domain
  moving bubble   the same bubble carried at u_y = V between  (Sec. 6.3)
                  a specular side and a moving wall
  phase separation between cold plates                      (Sec. 7)

Noise.  The paper draws U(-0.01, 0.01) per node on a grid of 320 nodes per
unit length (Sec. 7).  The surface energy of per-node noise grows like
1/ds^2, and on grids finer than ~256 per unit length it drives near-sonic
flow that leaves the model's range (measured: per-node noise at ds = 1/1024
diverges within 500 steps for any stable dt).  The noise is therefore drawn
per node of a grid with at most 256 nodes per unit length and Fourier-
interpolated to the full grid (``band_limited_noise``); on grids of at most
256 nodes per unit length it is plain per-node noise.

Time steps.  Besides the CFL rule p_max dt / ds < 1 (Sec. 4.1), the
capillary term sigma grad(Laplacian n) of Eq. F_def makes the step stiff:
the fastest mode along one axis has omega ~ 2.7 sqrt(sigma n) / ds^2, about
twice that along the grid diagonal, and RK-3 needs omega dt < sqrt(3)
(measured: at ds = 1/1024 the 2-D planar set-up diverges within 250 steps at
dt = 5e-5 and runs cleanly at dt = 2.5e-5).  The workloads take dt with
2-D omega dt <= ~1.4.

Random draws use numpy's PCG64 with seed 1702016900 + k, k the workload
number below, so every run of every leg sees the same values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

SEED_BASE = 1702016900
P_MAX = math.sqrt(5.0 + math.sqrt(10.0))  # largest Gauss-Hermite Q=5 root

# Coexisting vapour / liquid densities of the reduced van der Waals fluid
# (a = 9/8, b = 1/3) from the Maxwell equal-area construction; the tests
# check these constants against the oracle's Maxwell solver.
MAXWELL = {
    0.7: (0.1280223017, 2.1404425485),
    0.8: (0.2396669218, 1.9327058286),
    0.9: (0.4257416377, 1.6572702120),
}


@dataclass
class RunParams:
    nx: int
    ny: int
    ds: float
    dt: float
    tau: float
    a: float = 9.0 / 8.0
    b: float = 1.0 / 3.0
    sigma: float = 1e-4
    Tw: tuple = (1.0, 1.0)
    uw: tuple = (0.0, 0.0)
    side_x: int = 0     # 0 periodic, 1 diffuse walls, 2 specular, 3 specular x = 0 + diffuse wall x = 1
    side_y: int = 0     # 0 periodic, 2 specular
    steps: int = 1
    name: str = ""

    def as_dict(self):
        return asdict(self)

    @property
    def cfl(self) -> float:
        return P_MAX * self.dt / self.ds


def node_x(nx: int, ds: float) -> np.ndarray:
    return (np.arange(nx) + 0.5) * ds


def node_y(ny: int, ds: float) -> np.ndarray:
    return (np.arange(ny) + 0.5) * ds


def shear_wave(nx: int, ny: int, ds: float, n0=1.0, T0=1.1, u0=1e-3, V=0.0, m: int = 1):
    """Uniform n, T; u_y = u0 sin(2 pi m x); u_x = V."""
    x = node_x(nx, ds)
    n = np.full((ny, nx), float(n0))
    T = np.full((ny, nx), float(T0))
    ux = np.full((ny, nx), float(V))
    uy = np.tile(u0 * np.sin(2.0 * math.pi * m * x), (ny, 1))
    return n, ux, uy, T


def longitudinal_wave(nx: int, ny: int, ds: float, n0=1.0, T0=1.1, u0=1e-3, m: int = 1):
    """Uniform n, T; u_x = u0 sin(2 pi m x); u_y = 0."""
    x = node_x(nx, ds)
    n = np.full((ny, nx), float(n0))
    T = np.full((ny, nx), float(T0))
    ux = np.tile(u0 * np.sin(2.0 * math.pi * m * x), (ny, 1))
    uy = np.zeros((ny, nx))
    return n, ux, uy, T


def noisy_rest(nx: int, ny: int, seed: int, n0=1.0, amp=0.01, T0=1.0):
    """n = n0 + amp U(-1, 1) per node, u = 0, uniform T (Sec. 7 recipe)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n0 + amp * rng.uniform(-1.0, 1.0, size=(ny, nx))
    z = np.zeros((ny, nx))
    return n, z.copy(), z.copy(), np.full((ny, nx), float(T0))


def band_limited_noise(nx: int, ny: int, seed: int, factor: int) -> np.ndarray:
    """U(-1, 1) per node of a (ny/factor) x (nx/factor) grid, Fourier-
    interpolated (zero-padded spectrum) to ny x nx; factor 1 is plain
    per-node noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if factor <= 1:
        return rng.uniform(-1.0, 1.0, size=(ny, nx))
    cy, cx = max(1, ny // factor), max(1, nx // factor)
    C = np.fft.fft2(rng.uniform(-1.0, 1.0, size=(cy, cx)))
    P = np.zeros((ny, nx), dtype=complex)
    hy, hx = (cy + 1) // 2, (cx + 1) // 2
    ly, lx = cy - hy, cx - hx
    P[:hy, :hx] = C[:hy, :hx]
    if lx:
        P[:hy, nx - lx:] = C[:hy, hx:]
    if ly:
        P[ny - ly:, :hx] = C[hy:, :hx]
        if lx:
            P[ny - ly:, nx - lx:] = C[hy:, hx:]
    return np.real(np.fft.ifft2(P)) * (ny * nx) / (cy * cx)


def noise_factor(nx: int, ds: float) -> int:
    """Coarsening factor that keeps the noise at most 256 nodes per unit length."""
    per_unit = 1.0 / ds
    f = 1
    while per_unit / f > 256 and nx % (2 * f) == 0:
        f *= 2
    return f


def cold_rest(nx: int, ny: int, ds: float, seed: int, n0=1.0, amp=0.01, T0=1.0):
    """n = n0 + amp * band-limited noise, u = 0, uniform T (Sec. 7 recipe at
    the noise resolution described in the module docstring)."""
    n = n0 + amp * band_limited_noise(nx, ny, seed, noise_factor(nx, ds))
    z = np.zeros((ny, nx))
    return n, z.copy(), z.copy(), np.full((ny, nx), float(T0))


def laplace_drop(nx: int, ny: int, ds: float, R: float, T: float,
                 width: float = 0.02, centre=(0.5, 0.5)):
    """Liquid drop of radius R in vapour: n = n_g + (n_l - n_g)/2 (1 - tanh((r - R)/width))."""
    ng, nl = MAXWELL[round(T, 6)]
    x = node_x(nx, ds)
    y = node_y(ny, ds)
    X, Y = np.meshgrid(x, y)
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2)
    n = ng + 0.5 * (nl - ng) * (1.0 - np.tanh((r - R) / width))
    z = np.zeros((ny, nx))
    return n, z.copy(), z.copy(), np.full((ny, nx), float(T))


# ---------------------------------------------------------------- workloads

def shear_64x4() -> tuple:
    """Shear-wave decay, 64 x 4 periodic, unit box: n0 = 1, T0 = 1.1,
    u_y = 1e-3 sin(2 pi x), tau = 0.01, dt = 0.002, 200 RK-3 steps."""
    p = RunParams(nx=64, ny=4, ds=1.0 / 64, dt=0.002, tau=0.01, steps=200,
                  name="shear-wave 64x4 periodic")
    return p, shear_wave(64, 4, p.ds, 1.0, 1.1, 1e-3)


def planar_walls(nx: int = 1024, ny: int = 8, steps: int = 20000) -> tuple:
    """Planar liquid-vapour set-up between diffuse walls at x = 0, 1 (periodic
    y): T_w = 0.9, n = 1 + 0.01 (band-limited) noise, T0 = 1, tau = 0.005,
    dt = 2.5e-5 * 1024 / nx (CFL 0.073, 2-D omega dt ~ 1.4 at nx = 1024),
    sigma = 1e-4."""
    ds = 1.0 / nx
    p = RunParams(nx=nx, ny=ny, ds=ds, dt=2.5e-5 * 1024.0 / nx, tau=0.005,
                  Tw=(0.9, 0.9), side_x=1, steps=steps,
                  name=f"planar interface {nx}x{ny} diffuse walls")
    return p, cold_rest(nx, ny, ds, SEED_BASE + 1, 1.0, 0.01, 1.0)


def planar_tanh(nx: int = 320, Tw: float = 0.9, dt: float = 2e-4, steps: int = 100000, sigma: float = 1e-4,
                densities=None) -> tuple:
    """Liquid slabs at the diffuse walls x = 0, 1 and vapour in the middle
    (ny = 1, periodic y), the full-channel form of the paper's half-channel
    planar set-up (Sec. 4): n = n_g + (n_l - n_g)/2 [1 + tanh((|x - 1/2| -
    1/4) / xi)] (Eq. tanh, interfaces at 1/4 and 3/4), Maxwell densities at
    T = T_w, xi = sqrt(8 sigma / (9 (1 - T_w))) (Eq. xiwagner, sigma for its
    kappa), T = T_w, u = 0, tau = 0.005; ds = 1/320 and dt = 2e-4 as in the
    paper's planar runs.  `densities` = (n_g, n_l) for a T_w outside MAXWELL."""
    ds = 1.0 / nx
    ng, nl = densities if densities is not None else MAXWELL[round(Tw, 6)]
    xi = math.sqrt(8.0 * sigma / (9.0 * (1.0 - Tw)))
    x = node_x(nx, ds)
    n = ng + 0.5 * (nl - ng) * (1.0 + np.tanh((np.abs(x - 0.5) - 0.25) / xi))
    p = RunParams(nx=nx, ny=1, ds=ds, dt=dt, tau=0.005, sigma=sigma, Tw=(Tw, Tw), side_x=1, steps=steps,
                  name=f"planar tanh interfaces {nx}x1 diffuse walls Tw={Tw}")
    z = np.zeros((1, nx))
    return p, (n[None, :].copy(), z, z.copy(), np.full((1, nx), float(Tw)))


def laplace_bubble_quarter(R: float, sigma: float = 1e-4, Tw: float = 0.8, n: int = 160) -> tuple:
    """The paper's reduced Laplace domain (Sec. 5): x, y in [0, 1/2] with the
    channel centre at (0, 0), specular bottom, left and top sides and a
    diffuse wall at x = 1/2 (T_w); ds = 1/320, dt = 2e-4, tau = 5e-3.  A gas
    bubble of radius R centred at (0, 0): n = n_g + (n_l - n_g)/2 [1 +
    tanh((r - R) / xi)] with the Maxwell densities at T_w and xi of
    Eq. xiwagner, T = T_w, u = 0."""
    ds = 0.5 / n
    ng, nl = MAXWELL[round(Tw, 6)]
    xi = math.sqrt(8.0 * sigma / (9.0 * (1.0 - Tw)))
    x = node_x(n, ds)
    X, Y = np.meshgrid(x, x)
    r = np.sqrt(X ** 2 + Y ** 2)
    dens = ng + 0.5 * (nl - ng) * (1.0 + np.tanh((r - R) / xi))
    p = RunParams(nx=n, ny=n, ds=ds, dt=2e-4, tau=5e-3, sigma=sigma, Tw=(Tw, Tw), side_x=3, side_y=2,
                  name=f"Laplace bubble R={R} quarter domain {n}^2")
    z = np.zeros((n, n))
    return p, (dens, z, z.copy(), np.full((n, n), float(Tw)))


def moving_bubble(V: float, R: float = 0.25, sigma: float = 1e-4, Tw: float = 0.8) -> tuple:
    """The moving-bubble set-up of Sec. 6.3: x in [0, 1/2] with a specular
    side at x = 0 and a diffuse wall at x = 1/2 (T_w, moving along y at
    u_w = V), periodic y over a unit length (y in [-1/2, 1/2)); a gas bubble
    of radius R centred at (0, 0) (Eq. tanh, Maxwell densities at T_w, xi of
    Eq. xiwagner), T = T_w and u_y = V everywhere; ds = 1/320, dt = 2e-4,
    tau = 5e-3.  Node y-coordinates of the returned fields are
    node_y(ny, ds) - 1/2."""
    ds = 1.0 / 320
    nx, ny = 160, 320
    ng, nl = MAXWELL[round(Tw, 6)]
    xi = math.sqrt(8.0 * sigma / (9.0 * (1.0 - Tw)))
    X, Y = np.meshgrid(node_x(nx, ds), node_y(ny, ds) - 0.5)
    n = ng + 0.5 * (nl - ng) * (1.0 + np.tanh((np.sqrt(X ** 2 + Y ** 2) - R) / xi))
    p = RunParams(nx=nx, ny=ny, ds=ds, dt=2e-4, tau=5e-3, sigma=sigma, Tw=(Tw, Tw), uw=(V, V), side_x=3, side_y=0,
                  name=f"moving bubble V={V}")
    return p, (n, np.zeros_like(n), np.full_like(n, float(V)), np.full_like(n, float(Tw)))


def laplace(n: int = 2048, R: float = 0.2, steps: int = 5000) -> tuple:
    """Laplace drop on an n x n periodic grid, T = 0.9, tanh width 0.02,
    dt = 2.5e-6 (2048 / n)^2 (capillary limit, 2-D omega dt ~ 0.7; CFL 0.015
    at n = 2048), tau = 5e-3, sigma = 1e-4."""
    ds = 1.0 / n
    p = RunParams(nx=n, ny=n, ds=ds, dt=2.5e-6 * (2048.0 / n) ** 2, tau=5e-3,
                  steps=steps, name=f"Laplace drop {n}^2 R={R}")
    return p, laplace_drop(n, n, ds, R, 0.9)


def phase_separation(n: int = 4096, Tw: float = 0.7, steps: int = 10000) -> tuple:
    """Phase separation between cold plates (Sec. 7 set-up): n x n, diffuse
    walls at x = 0, 1, periodic y, T_w = 0.7, n = 1 + 0.01 (band-limited)
    noise, T0 = 1, dt = 6.25e-7 (4096 / n)^2 (capillary limit, 2-D omega dt
    ~ 0.7; CFL 0.007 at n = 4096), tau = 5e-3, sigma = 1e-4."""
    ds = 1.0 / n
    p = RunParams(nx=n, ny=n, ds=ds, dt=6.25e-7 * (4096.0 / n) ** 2, tau=5e-3,
                  Tw=(Tw, Tw), side_x=1, steps=steps,
                  name=f"phase separation {n}^2 Tw={Tw}")
    return p, cold_rest(n, n, ds, SEED_BASE + 5, 1.0, 0.01, 1.0)


def stable_dt(ds: float, sigma: float = 1e-4, n_max: float = 1.0, cfl: float = 0.146,
              omega_dt: float = 0.7) -> float:
    """Largest dt with p_max dt / ds <= cfl and 2-D capillary omega dt <= omega_dt
    (omega ~ 2 x 2.7 sqrt(sigma n_max) / ds^2, see the module docstring)."""
    dt = cfl * ds / P_MAX
    if sigma > 0:
        dt = min(dt, omega_dt / (5.4 * math.sqrt(sigma * n_max) / ds ** 2))
    return dt


def batch_sweep(max_n: int = 1024) -> list:
    """The 64 independent runs of the batched workload (sizes capped at max_n):
    22 shear waves (N in 32 .. 1024, T0 = 0.8 and 1.1), 11 longitudinal waves
    (T0 = 1.1), 15 Laplace drops (R = 0.1 .. 0.3 on 256^2 .. 1024^2, T = 0.9)
    and 16 planar wall runs (T_w = 0.75 .. 0.9 on nx = 256 .. 2048, ny = 8);
    amplitude 1e-3, tau = 0.01 for the waves, dt = stable_dt per run."""
    runs = []
    sizes = [min(n, max_n) for n in (32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024)]
    for T0 in (0.8, 1.1):
        for N in sizes:
            ds = 1.0 / N
            p = RunParams(nx=N, ny=N, ds=ds, dt=stable_dt(ds), tau=0.01, name=f"shear {N}^2 T0={T0}")
            runs.append((p, shear_wave(N, N, ds, 1.0, T0, 1e-3)))
    for N in sizes:
        ds = 1.0 / N
        p = RunParams(nx=N, ny=N, ds=ds, dt=stable_dt(ds), tau=0.01, name=f"longitudinal {N}^2")
        runs.append((p, longitudinal_wave(N, N, ds, 1.0, 1.1, 1e-3)))
    for R in (0.1, 0.15, 0.2, 0.25, 0.3):
        for N in (256, 512, 1024):
            N = min(N, max_n)
            ds = 1.0 / N
            p = RunParams(nx=N, ny=N, ds=ds, dt=stable_dt(ds, n_max=1.66), tau=5e-3, name=f"Laplace {N}^2 R={R}")
            runs.append((p, laplace_drop(N, N, ds, R, 0.9)))
    for Tw in (0.75, 0.8, 0.85, 0.9):
        for nx in (256, 512, 1024, 2048):
            nx = min(nx, 2 * max_n)
            ds = 1.0 / nx
            p = RunParams(nx=nx, ny=8, ds=ds, dt=stable_dt(ds, n_max=2.2), tau=0.005, Tw=(Tw, Tw), side_x=1,
                          name=f"planar {nx}x8 Tw={Tw}")
            runs.append((p, cold_rest(nx, 8, ds, SEED_BASE + 4, 1.0, 0.01, 1.0)))
    return runs
