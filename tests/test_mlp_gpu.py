"""Learned WENO-5 weights: the GPU network against the FP64 oracle network
(forward, gradient), GPU training, the learned stage kernel against the
oracle's learned mode, and what the trained network gains over WENO-5-JS."""
import math

import numpy as np
import pytest

import oracle
from helpers import make_oracle, moments_rel
from oracle import analytic, mlp
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


def learned_face_values(olb, theta, V):
    """Interface values of stencils V [S][5] with the weights of the library's
    network (olb_mlp_forward on the GPU), combined with the candidates on the
    host; Jiang-Shu values (Table tab:weno) where the network does not act."""
    V = np.asarray(V, dtype=np.float64)
    X, _ = mlp.normalise(V)
    w = olb.mlp_forward(theta, X.astype(np.float32)).cpu().numpy().astype(np.float64)
    out = V[:, 2] + (w * mlp.candidates(V)).sum(axis=1)
    js = ~mlp.network_acts(V)
    out[js] = mlp.js_face_values(V[js])
    return out


def random_samples(S, seed=0):
    rng = np.random.default_rng(seed)
    V = rng.normal(size=(S, 5)).cumsum(axis=1)
    X, r = mlp.normalise(V)
    Gn = mlp.candidates(V) / r[:, None]
    tn = rng.normal(scale=0.2, size=S)
    return X.astype(np.float32), Gn.astype(np.float32), tn.astype(np.float32)


def test_forward_matches_oracle(olb):
    theta = mlp.init_params(1).astype(np.float32)
    X, _, _ = random_samples(3000, 2)
    w = olb.mlp_forward(theta, X).cpu().numpy()
    ref, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(w - ref)) < 2e-6


def test_gradient_matches_oracle(olb):
    """GPU backward (FP32, per-CTA sums) against the FP64 oracle gradient,
    itself pinned by central finite differences."""
    theta = mlp.init_params(3).astype(np.float32)
    X, Gn, tn = random_samples(5000, 4)
    loss, g = olb.mlp_grad(theta, X, Gn, tn)
    g = g.cpu().numpy()
    t64 = theta.astype(np.float64)
    ref_loss = mlp.loss(t64, X.astype(np.float64), Gn.astype(np.float64), tn.astype(np.float64))
    ref = mlp.grad(t64, X.astype(np.float64), Gn.astype(np.float64), tn.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-5 * ref_loss
    assert np.linalg.norm(g - ref) < 1e-4 * np.linalg.norm(ref)


@pytest.fixture(scope="module")
def trained(olb):
    """Network trained on the GPU on 80 % of the stencils harvested from solver
    runs; the other 20 % (never seen in training) are kept for evaluation."""
    from paper_1702_01690_gb300 import learned
    V, t, s = learned.harvest(learned.default_sources(), ratio=4, row_stride=16)
    (x, Gn, tn), (Vk, tk, rk) = learned.normalised_samples(V, t, s)
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(tn))
    cut = int(0.8 * len(tn))
    tr, te = perm[:cut], perm[cut:]
    theta, hist = learned.train(x[tr], Gn[tr], tn[tr], epochs=30, batch=4096, lr=2e-3)
    return theta, hist, len(tr), (Vk[te], tk[te], rk[te]), (Vk[tr], tk[tr], rk[tr])


def test_training_reduces_loss(olb, trained):
    """Training lowers the loss, and below the loss the Jiang-Shu weights give
    on the training stencils."""
    theta, hist, n, _, (V, t, r) = trained
    js = np.mean(((mlp.js_face_values(V) - t) / r) ** 2)
    ours = np.mean(((learned_face_values(olb, theta, V) - t) / r) ** 2)
    print("samples", n, "loss per epoch", hist, "JS loss", js, "trained loss", ours)
    assert n > 10000
    assert hist[-1] < hist[0]
    assert ours < js


def test_trained_network_gains_over_js(olb, trained):
    """Interface error against the fine-grid targets on stencils never seen in
    training (held-out 20 % of the same runs): the learned weights beat
    Jiang-Shu's.  On runs not used at all (another drop radius, another wave
    amplitude) the error stays within 1.5 x Jiang-Shu's.  The network's
    weights come from the library (olb_mlp_forward)."""
    from paper_1702_01690_gb300 import learned
    theta, _, _, (V, t, r), _ = trained
    e_js = np.sqrt(np.mean(((mlp.js_face_values(V) - t) / r) ** 2))
    e_l = np.sqrt(np.mean(((learned_face_values(olb, theta, V) - t) / r) ** 2))
    print(f"held-out stencils: JS {e_js:.3e}  learned {e_l:.3e}  ratio {e_l / e_js:.3f}")
    assert e_l < e_js
    held = []
    p, f = inputs.laplace(512, R=0.25, steps=4)
    held.append((p, f, 4))
    ds = 1.0 / 256
    p = inputs.RunParams(nx=256, ny=256, ds=ds, dt=inputs.stable_dt(ds), tau=0.01)
    held.append((p, inputs.shear_wave(256, 256, ds, 1.0, 0.9, 0.1), 4))
    V, t, s = learned.harvest(held, ratio=4, row_stride=16)
    (_, _, _), (V, t, r) = learned.normalised_samples(V, t, s)
    e_js = np.sqrt(np.mean(((mlp.js_face_values(V) - t) / r) ** 2))
    e_l = np.sqrt(np.mean(((learned_face_values(olb, theta, V) - t) / r) ** 2))
    print(f"held-out runs: JS {e_js:.3e}  learned {e_l:.3e}  ratio {e_l / e_js:.3f}")
    assert e_l <= 1.5 * e_js


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_stage_matches_oracle(olb, trained, precision):
    """The learned stage kernel against the oracle's learned mode (FP64
    network) after 5 steps of a noisy wall run: FP64 path within 1e-6 on
    n, u, T (the GPU network runs in FP32); FP32 path within 1e-5."""
    theta = trained[0]
    p, _ = inputs.planar_walls(nx=48, ny=16)
    n, ux, uy, T = inputs.noisy_rest(48, 16, 21, 1.0, 0.02, 0.95)
    fl = (n, 0.01 * np.sin(np.arange(48) / 5.0)[None, :] + 0 * n, uy, T)
    ctx = olb.create(p, precision, weno_mode=olb.WENO_LEARNED)
    with pytest.raises(olb.OlbError):
        ctx.init_fields(*fl)
        ctx.step(1)  # network not loaded yet
    ctx.set_weno_mlp(theta)
    ctx.init_fields(*fl)
    assert ctx.step(5) == 0
    o = make_oracle(p, fl)
    o.set_mlp(theta.astype(np.float64))
    o.step(5)
    err = moments_rel(ctx.moments(), o.moments())
    print("learned stage vs oracle", precision, err)
    assert max(err.values()) < (1e-6 if precision == 0 else 1e-5), err


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_stage_every_shape_identical(olb, trained, precision):
    """The learned stage on every shape it is compiled for, (8,8,4),
    (16,8,2), (32,16,1), on a 70 x 37 wall grid (ragged tiles of every
    shape): populations bit for bit equal; the large-tile run against the
    oracle's learned mode."""
    theta = trained[0]
    p = inputs.RunParams(nx=70, ny=37, ds=1.0 / 70, dt=0.2 / 70 / inputs.P_MAX, tau=0.01,
                         Tw=(0.85, 0.95), uw=(0.01, -0.02), side_x=1)
    rng = np.random.default_rng(70)
    n = 1.0 + 0.05 * rng.uniform(-1, 1, (37, 70))
    ux, uy = 0.01 * rng.uniform(-1, 1, (2, 37, 70))
    fl = (n, ux, uy, np.full((37, 70), 0.95))
    ref = None
    for shape in ((8, 8, 4), (16, 8, 2), (32, 16, 1)):
        ctx = olb.create(p, precision, weno_mode=olb.WENO_LEARNED)
        ctx.set_tile(*shape)
        ctx.set_weno_mlp(theta)
        ctx.init_fields(*fl)
        assert ctx.step(4) == 0
        f = ctx.get_populations()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref), shape
    o = make_oracle(p, fl)
    o.set_mlp(theta.astype(np.float64))
    o.step(4)
    err = moments_rel(ctx.moments(), o.moments())
    assert max(err.values()) < (1e-6 if precision == 0 else 1e-5), err


def test_learned_solver_accuracy_and_order(olb, trained):
    """Shear wave (T0 = 0.8, tau = 0.01) in FP64 with the learned weights:
    the amplitude error against a fine reference at N = 16, 32, 64 stays
    within 1.5 x the WENO-5-JS error, and the order between N = 32 and 64
    stays >= 4."""
    theta = trained[0]

    def amp(N, learned_mode):
        ds = 1.0 / N
        p = inputs.RunParams(nx=N, ny=1, ds=ds, dt=1.25e-4, tau=0.01)
        from paper_1702_01690_gb300 import olb as o
        ctx = o.create(p, o.FP64, weno_mode=o.WENO_LEARNED if learned_mode else o.WENO_JS)
        if learned_mode:
            ctx.set_weno_mlp(theta)
        ctx.init_fields(*inputs.shear_wave(N, 1, ds, 1.0, 0.8, 1e-3))
        ctx.step(400)
        return analytic.shear_amplitude(ctx.moments()[2], inputs.node_x(N, ds), 2 * math.pi)

    ref = amp(256, False)
    errs = {m: [abs(amp(N, m) - ref) for N in (16, 32, 64)] for m in (False, True)}
    print("amplitude errors JS", errs[False], "learned", errs[True])
    for k in range(3):
        assert errs[True][k] <= 1.5 * errs[False][k]
    order = math.log2(errs[True][1] / errs[True][2])
    assert order >= 4.0, order
