"""The WENO-5 forms that the stage kernel evaluates, checked symbolically
against the paper's definitions (Sec. 3.2, Eqs. weno5_flux, weno5_omega,
weno5_delta, weno5_sigma).

The kernel (csrc/olb_kernels.cuh, weno5_core) writes the smoothness
indicators as quadratic forms in the first differences d01 = v1 - v0, ...,
d34 = v4 - v3 (the middle one factored as d12 (d12 - 5/4 d23) + d23^2), the
candidates as 6 (F^q - v2), and the Jiang-Shu weights in product form with a
single normalisation.  These tests restate those forms and the paper's and
show that they agree exactly, up to the common factors that the normalised
weights do not see.  (The GPU parity tests compare the kernel's numbers with
the oracle; this checks the algebra behind the rewrite on the CPU.)
"""
import numpy as np
import pytest

sp = pytest.importorskip("sympy")

v0, v1, v2, v3, v4 = sp.symbols("v0:5", real=True)
d01, d12, d23, d34 = v1 - v0, v2 - v1, v3 - v2, v4 - v3


def paper_indicators():
    # f_{i-2} .. f_{i+2} = v0 .. v4 (upwind orientation)
    s1 = sp.Rational(13, 12) * (v0 - 2 * v1 + v2) ** 2 + sp.Rational(1, 4) * (v0 - 4 * v1 + 3 * v2) ** 2
    s2 = sp.Rational(13, 12) * (v1 - 2 * v2 + v3) ** 2 + sp.Rational(1, 4) * (v1 - v3) ** 2
    s3 = sp.Rational(13, 12) * (v2 - 2 * v3 + v4) ** 2 + sp.Rational(1, 4) * (3 * v2 - 4 * v3 + v4) ** 2
    return s1, s2, s3


def kernel_indicators():
    s1 = d01 * (d01 - sp.Rational(11, 4) * d12) + sp.Rational(5, 2) * d12 ** 2
    s2 = d12 * (d12 - sp.Rational(5, 4) * d23) + d23 ** 2
    s3 = d34 * (d34 - sp.Rational(11, 4) * d23) + sp.Rational(5, 2) * d23 ** 2
    return s1, s2, s3


def paper_candidates():
    F1 = sp.Rational(1, 3) * v0 - sp.Rational(7, 6) * v1 + sp.Rational(11, 6) * v2
    F2 = -sp.Rational(1, 6) * v1 + sp.Rational(5, 6) * v2 + sp.Rational(1, 3) * v3
    F3 = sp.Rational(1, 3) * v2 + sp.Rational(5, 6) * v3 - sp.Rational(1, 6) * v4
    return F1, F2, F3


def kernel_candidates():
    return 5 * d12 - 2 * d01, d12 + 2 * d23, 4 * d23 - d34


def test_indicators_are_the_papers_times_twelve_sixteenths():
    for paper, kernel in zip(paper_indicators(), kernel_indicators()):
        assert sp.expand(sp.Rational(12, 16) * paper - kernel) == 0


def test_candidates_are_six_times_the_papers_relative_to_the_middle_node():
    for paper, kernel in zip(paper_candidates(), kernel_candidates()):
        assert sp.expand(6 * (paper - v2) - kernel) == 0


def test_product_form_weights_and_face_value_equal_the_papers():
    """A_q = c_q prod_{r != q} s_r^2 with (c_1, c_2, c_3) = (1, 6, 3) = 10
    delta_q, normalised once, gives the paper's weights, and v2 + sum A_q G_q /
    (6 sum A_q) is the paper's sum_q wbar_q F^q (p/m = 1).  Checked as a
    rational identity in the indicator values and at random stencils."""
    S1, S2, S3 = sp.symbols("S1:4", positive=True)
    delta = (sp.Rational(1, 10), sp.Rational(6, 10), sp.Rational(3, 10))
    # weights as functions of the indicator values
    wt = [d / s ** 2 for d, s in zip(delta, (S1, S2, S3))]
    wbar = [w / sum(wt) for w in wt]
    A = [(S2 * S3) ** 2, 6 * (S1 * S3) ** 2, 3 * (S1 * S2) ** 2]
    for q in range(3):
        assert sp.simplify(A[q] / sum(A) - wbar[q]) == 0
    # the same weights with the kernel's indicators (a common factor 12/16 apart)
    rng = np.random.default_rng(3)
    sub_k = dict(zip((S1, S2, S3), kernel_indicators()))
    sub_p = dict(zip((S1, S2, S3), paper_indicators()))
    face_kernel = v2 + sum(a * g for a, g in zip(A, kernel_candidates())) / (6 * sum(A))
    face_paper = sum(w * F for w, F in zip(wbar, paper_candidates()))
    for _ in range(20):
        vals = {v: sp.Rational(int(x), 97) for v, x in zip((v0, v1, v2, v3, v4), rng.integers(-300, 300, 5))}
        k = face_kernel.subs(sub_k).subs(vals)
        p = face_paper.subs(sub_p).subs(vals)
        if any(s.subs(vals) == 0 for s in paper_indicators()):
            continue  # a vanishing indicator takes Table tab:weno (tested on the oracle side)
        assert sp.simplify(k - p) == 0


def test_strip_recurrence_carries_the_next_faces_differences():
    """In a strip the next face's stencil is the current one shifted by one
    node downwind: its d01, d12, d23 are the current d12, d23, d34 and its
    scaled square 2.5 d12^2 is the current 2.5 d23^2, so carrying them gives
    the same operands as recomputing them."""
    w = sp.symbols("w", real=True)  # the new downwind value
    nd01, nd12, nd23, nd34 = v2 - v1, v3 - v2, v4 - v3, w - v4
    assert sp.expand(nd01 - d12) == 0 and sp.expand(nd12 - d23) == 0 and sp.expand(nd23 - d34) == 0
    assert sp.expand(sp.Rational(5, 2) * nd12 ** 2 - sp.Rational(5, 2) * d23 ** 2) == 0
