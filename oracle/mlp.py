"""FP64 reference of the learned WENO-5 weight network (test infrastructure).

A small MLP stands in for the non-linear weight step of WENO-5 (Eq.
weno5_omega): it maps the five stencil values of an interface, normalised as
x = (v - mean v) / (max v - min v) (invariant to shifts and scales of f, like
the Jiang-Shu weights), to three convex weights:

    h1 = tanh(W1 x + b1)      (32)
    h2 = tanh(W2 h1 + b2)     (32)
    w  = softmax(W3 h2 + b3)  (3)

Parameter vector (1347 values, the layout the library's olb_mlp_* calls
document): W1 [32][5], b1 [32], W2 [32][32], b2 [32], W3 [3][32], b3 [3],
row-major, concatenated.

The network acts only where the stencil is not smooth in the Jiang-Shu sense
(min sigma_q < 0.9 max sigma_q, sigma_q of Eq. weno5_sigma) and no indicator
vanishes; elsewhere the Jiang-Shu weights apply (guard()).

Training objective: the interface value v2 + sum_q w_q G_q (G_q the candidate
values minus v2, Eq. weno5_flux) should match a target t; in normalised units
the per-sample loss is (sum_q w_q G_q / r - (t - v2) / r)^2, r = max - min,
averaged over the samples.  forward/loss/grad below are plain numpy; grad is
pinned against central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 5, 32, 3
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            parts.append(rng.uniform(-lim, lim, shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts)


def normalise(V):
    """Stencils V [S][5] -> x [S][5] and range r [S] (r = 0 rows give x = 0)."""
    V = np.asarray(V, dtype=np.float64)
    r = V.max(axis=1) - V.min(axis=1)
    rs = np.where(r > 0, r, 1.0)
    return (V - V.mean(axis=1, keepdims=True)) / rs[:, None], r


def candidates(V):
    """G_q = F^q - v2 of Eq. weno5_flux for stencils V [S][5] (upwind order)."""
    V = np.asarray(V, dtype=np.float64)
    v0, v1, v2, v3, v4 = V.T
    F1 = v0 / 3 - 7 * v1 / 6 + 11 * v2 / 6
    F2 = -v1 / 6 + 5 * v2 / 6 + v3 / 3
    F3 = v2 / 3 + 5 * v3 / 6 - v4 / 6
    return np.stack([F1 - v2, F2 - v2, F3 - v2], axis=1)


def forward(theta, X):
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.tanh(a2)
    z = h2 @ P["W3"].T + P["b3"]
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    w = e / e.sum(axis=1, keepdims=True)
    return w, (X, h1, h2, w)


def loss(theta, X, Gn, tn):
    """Mean over samples of (sum_q w_q Gn_q - tn)^2 (normalised units)."""
    w, _ = forward(theta, X)
    res = (w * Gn).sum(axis=1) - tn
    return float(np.mean(res ** 2))


def grad(theta, X, Gn, tn):
    """Gradient of loss() by hand-written backpropagation."""
    P = unpack(theta)
    w, (X, h1, h2, _) = forward(theta, X)
    S = X.shape[0]
    res = (w * Gn).sum(axis=1) - np.asarray(tn)
    dw = (2.0 / S) * res[:, None] * Gn                     # dL/dw
    dz = w * (dw - (w * dw).sum(axis=1, keepdims=True))    # softmax backward
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    da2 = (dz @ P["W3"]) * (1.0 - h2 ** 2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ P["W2"]) * (1.0 - h1 ** 2)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def face_values(theta, V):
    """Learned interface values v2 + sum_q w_q G_q of stencils V [S][5]."""
    X, _ = normalise(V)
    w, _ = forward(theta, X)
    return np.asarray(V)[:, 2] + (w * candidates(V)).sum(axis=1)


GUARD = 0.9


def sigmas(V):
    """Smoothness indicators of Eq. weno5_sigma of stencils V [S][5]."""
    V = np.asarray(V, dtype=np.float64)
    v0, v1, v2, v3, v4 = V.T
    s1 = 13 / 12 * (v0 - 2 * v1 + v2) ** 2 + 0.25 * (v0 - 4 * v1 + 3 * v2) ** 2
    s2 = 13 / 12 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - v3) ** 2
    s3 = 13 / 12 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (3 * v2 - 4 * v3 + v4) ** 2
    return np.stack([s1, s2, s3], axis=1)


def network_acts(V):
    """Rows where the network's weights are used: no vanishing indicator and
    min sigma < GUARD max sigma."""
    S = sigmas(V)
    return (S.min(axis=1) > 0) & (S.min(axis=1) < GUARD * S.max(axis=1))


def js_face_values(V):
    """Jiang-Shu WENO-5 interface values of stencils V [S][5] (upwind order):
    Eq. weno5_omega without epsilon, Table tab:weno where an indicator
    vanishes (the same reading as orc_weno5, vectorised for many stencils)."""
    V = np.asarray(V, dtype=np.float64)
    S = sigmas(V)
    d = np.array([0.1, 0.6, 0.3])
    zero = S == 0
    anyz = zero.any(axis=1)
    Sn = np.where(zero, 1.0, S)
    wt = np.where(anyz[:, None], d * zero, d / Sn ** 2)
    wt = wt / wt.sum(axis=1, keepdims=True)
    return V[:, 2] + (wt * candidates(V)).sum(axis=1)
