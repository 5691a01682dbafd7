"""The learned-weight guard's FP32 pre-check (csrc/olb_mlp.cuh, learned_guard).

The guard hands a stencil to the network when no smoothness indicator
vanishes and min sigma_q < 0.9 max sigma_q (Sec. 3.2's indicators, in the
kernel's form sigma_q = 13 a_q^2 + 3 b_q^2 with a_q, b_q first-difference
combinations).  In the FP64 kernel it first decides from the differences
rounded to FP32 and falls back to FP64 within a relative band of 1e-4 around
the threshold.  That is sound because each sigma_q is a positive-definite
quadratic form in two differences: the FP32 values carry a relative error of
a few 1e-6.  These tests emulate the FP32 arithmetic with numpy and check, on
stencils spread over magnitudes and packed near the threshold, that every
decision the pre-check takes is the one the FP64 comparison takes.  They also
check the exact zero test on the differences' bits against the FP64 one on
a_q, b_q.  CPU only.
"""
import numpy as np

GUARD = 0.9


def _fma32(a, b, c):
    # FP32 fused multiply-add: the FP32 product is exact in FP64 (48 bits),
    # the sum is rounded once to FP64 and then to FP32 (a double rounding that
    # is at most one FP32 ulp from the single one, far inside the band)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _forms(d01, d12, d23, d34, dtype):
    """a_q, b_q and sigma_q as the kernel evaluates them, in dtype."""
    f = (lambda a, b, c: _fma32(a, b, c)) if dtype == np.float32 else (lambda a, b, c: a * b + c)
    t = lambda v: np.asarray(v, dtype=dtype)  # noqa: E731
    d01, d12, d23, d34 = t(d01), t(d12), t(d23), t(d34)
    a1, b1 = d12 - d01, f(t(3.0) * np.ones_like(d12), d12, -d01)
    a2, b2 = d23 - d12, d12 + d23
    a3, b3 = d34 - d23, f(t(-3.0) * np.ones_like(d23), d23, d34)
    sig = [f(t(13.0) * a, a, (t(3.0) * b) * b) for a, b in ((a1, b1), (a2, b2), (a3, b3))]
    return (a1, b1, a2, b2, a3, b3), sig


def _precheck(d):
    """The FP32 pre-check: True (network), False (Jiang-Shu) or None (FP64 decides)."""
    _, (f1, f2, f3) = _forms(*(x.astype(np.float32) for x in d), np.float32)
    mn = np.minimum(f1, np.minimum(f2, f3))
    mx = np.maximum(f1, np.maximum(f2, f3))
    ok = (mx > np.float32(1e-30)) & (mx < np.float32(1e30))
    lo = np.float32(GUARD * (1.0 - 1e-4)) * mx
    hi = np.float32(GUARD * (1.0 + 1e-4)) * mx
    out = np.full(mn.shape, -1, dtype=np.int8)
    out[ok & (mn < lo)] = 1
    out[ok & ~(mn < lo) & (mn > hi)] = 0
    return out


def _fp64_decision(d):
    _, (s1, s2, s3) = _forms(*d, np.float64)
    mn = np.minimum(s1, np.minimum(s2, s3))
    mx = np.maximum(s1, np.maximum(s2, s3))
    return mn < GUARD * mx


def _stencils(rng, n):
    base = rng.standard_normal((4, n))
    scale = 10.0 ** rng.uniform(-14, 4, n)
    return base * scale


def _near_threshold(rng, n):
    """Stencils whose indicator ratio lies within ~1e-3 of the threshold: start
    from random differences and move d34 along sigma_3 until min/max = 0.9."""
    d = rng.standard_normal((4, n))
    out = []
    for k in range(n):
        d01, d12, d23 = d[0, k], d[1, k], d[2, k]
        s1 = 13 * (d12 - d01) ** 2 + 3 * (3 * d12 - d01) ** 2
        s2 = 13 * (d23 - d12) ** 2 + 3 * (d12 + d23) ** 2
        target = GUARD * max(s1, s2) if min(s1, s2) >= GUARD * max(s1, s2) else None
        if target is None:
            continue
        # sigma_3(d34) = 13 (d34 - d23)^2 + 3 (d34 - 3 d23)^2 = target, solved for d34
        A, B, C = 16.0, -(26 * d23 + 18 * d23), 13 * d23 ** 2 + 27 * d23 ** 2 - target
        disc = B * B - 4 * A * C
        if disc < 0:
            continue
        d34 = (-B + np.sqrt(disc)) / (2 * A)
        for eps in (-1e-3, -1e-5, -1e-7, 0.0, 1e-7, 1e-5, 1e-3):
            out.append((d01, d12, d23, d34 * (1 + eps)))
    arr = np.array(out).T
    return arr * 10.0 ** rng.uniform(-10, 3, arr.shape[1])


def test_precheck_decisions_match_fp64():
    rng = np.random.default_rng(20260601)
    for d in (_stencils(rng, 400_000), _near_threshold(rng, 20_000)):
        pre = _precheck(d)
        ref = _fp64_decision(d)
        decided = pre >= 0
        assert np.array_equal(pre[decided] == 1, ref[decided])
        # the band leaves almost every random stencil to the FP32 test
        if d.shape[1] == 400_000:
            assert decided.mean() > 0.999


def test_near_threshold_cases_reach_the_fp64_fallback():
    rng = np.random.default_rng(7)
    d = _near_threshold(rng, 5_000)
    pre = _precheck(d)
    assert (pre < 0).sum() > 0  # the band is exercised
    ref = _fp64_decision(d)
    decided = pre >= 0
    assert np.array_equal(pre[decided] == 1, ref[decided])


def test_zero_test_on_differences_equals_the_one_on_a_and_b():
    """a_q = b_q = 0 exactly when both differences of sub-stencil q are 0."""
    rng = np.random.default_rng(11)
    vals = np.array([0.0, -0.0, 1e-300, -1e-300, 5e-324, 1.0, 3.0, -2.5, 1e-17, 3e-17])
    d = rng.choice(vals, size=(4, 20_000))
    (a1, b1, a2, b2, a3, b3), _ = _forms(*d, np.float64)
    z_ab = ((a1 == 0) & (b1 == 0)) | ((a2 == 0) & (b2 == 0)) | ((a3 == 0) & (b3 == 0))
    z_d = ((d[0] == 0) & (d[1] == 0)) | ((d[1] == 0) & (d[2] == 0)) | ((d[2] == 0) & (d[3] == 0))
    assert np.array_equal(z_ab, z_d)
