"""Pins of the FP64 reference of the learned WENO weight network (CPU)."""
import numpy as np
import pytest

import oracle
from oracle import mlp


def data(S=64, seed=0):
    rng = np.random.default_rng(seed)
    V = rng.normal(size=(S, 5)).cumsum(axis=1)
    X, r = mlp.normalise(V)
    G = mlp.candidates(V) / r[:, None]
    t = rng.normal(scale=0.3, size=S)
    return V, X, G, t


def test_parameter_count():
    assert mlp.N_PARAMS == 5 * 32 + 32 + 32 * 32 + 32 + 3 * 32 + 3 == 1347


def test_grad_matches_central_differences():
    theta = mlp.init_params(1)
    _, X, G, t = data()
    g = mlp.grad(theta, X, G, t)
    rng = np.random.default_rng(2)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(theta + e, X, G, t) - mlp.loss(theta - e, X, G, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_weights_are_convex():
    theta = mlp.init_params(3)
    _, X, _, _ = data()
    w, _ = mlp.forward(theta, X)
    assert np.all(w > 0) and np.allclose(w.sum(axis=1), 1.0, atol=1e-15)


def test_ideal_weight_network_is_the_linear_5th_order_scheme():
    """With W3 = 0 and b3 = log(delta) the network returns the ideal weights
    (1/10, 6/10, 3/10) of Eq. weno5_delta: the face value is the linear
    5th-order upwind combination (2, -13, 47, 27, -3)/60."""
    theta = np.zeros(mlp.N_PARAMS)
    theta[1344:1347] = np.log([0.1, 0.6, 0.3])
    V, _, _, _ = data(400)
    # plus samples of smooth functions, on which the Jiang-Shu weights apply
    rng = np.random.default_rng(9)
    k = rng.uniform(0.01, 0.1, 200)[:, None]
    V = np.concatenate([V, np.sin(k * np.arange(5) + rng.uniform(0, 6.3, 200)[:, None])])
    ref = V @ np.array([2, -13, 47, 27, -3]) / 60.0
    np.testing.assert_allclose(mlp.face_values(theta, V), ref, rtol=1e-13, atol=1e-13)
    acts = mlp.network_acts(V)
    assert acts.sum() > 20 and (~acts).sum() > 20
    for v, a in zip(V, acts):
        expect = v @ np.array([2, -13, 47, 27, -3]) / 60.0 if a else oracle.weno5(v)
        assert abs(oracle.weno5_learned(theta, v) - expect) < 1e-13


def test_c_forward_matches_numpy():
    """The oracle's learned face value: the numpy network where it acts
    (min sigma < 0.9 max sigma), the Jiang-Shu value elsewhere."""
    theta = mlp.init_params(4)
    V, _, _, _ = data(200, 5)
    ref = mlp.face_values(theta, V)
    acts = mlp.network_acts(V)
    got = np.array([oracle.weno5_learned(theta, v) for v in V])
    js = np.array([oracle.weno5(v) for v in V])
    np.testing.assert_allclose(got[acts], ref[acts], rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(got[~acts], js[~acts])


def test_vanishing_indicator_falls_back_to_table():
    theta = mlp.init_params(6)
    for v in ([2.0, 2.0, 2.0, 1.1, 0.3], [1.3, 2.0, 2.0, 2.0, 2.0], [2.0] * 5):
        assert oracle.weno5_learned(theta, v) == oracle.weno5(v)


def test_learned_weights_shift_and_scale_invariant():
    theta = mlp.init_params(7)
    V, _, _, _ = data(16, 8)
    for v in V:
        _, w1 = oracle.weno5_learned(theta, v, return_weights=True)
        _, w2 = oracle.weno5_learned(theta, 4.0 * v - 1.5, return_weights=True)
        np.testing.assert_allclose(w1, w2, rtol=1e-12)


def test_vectorised_js_values_equal_the_c_oracle():
    """mlp.js_face_values (many stencils at once) against orc_weno5, itself
    pinned by Table tab:weno and exactness on quadratics: random stencils,
    stencils with one, two or three vanishing indicators."""
    rng = np.random.default_rng(5)
    V = list(rng.normal(size=(200, 5)).cumsum(axis=1))
    V += [np.array([1.0, 1.0, 1.0, 2.0, 4.0]), np.array([0.0, 1.0, 2.0, 3.0, 4.0]),
          np.array([3.0, 3.0, 3.0, 3.0, 3.0]), np.array([1.0, 2.0, 3.0, 3.0, 3.0]),
          np.array([5.0, 1.0, 2.0, 3.0, 4.0])]
    V = np.array(V)
    ref = np.array([oracle.weno5(v) for v in V])
    got = mlp.js_face_values(V)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
