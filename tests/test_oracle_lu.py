"""Pins of the oracle's pivoted LU and of the normalized power iterations
(Algorithm norm_iterations, Sec. 2.2.2) against library routines and facts
fixed by the mathematics."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1608_02148_gb300 import inputs
from tests.helpers import sin_theta


@pytest.mark.parametrize("m,l,seed", [(50, 7, 1), (300, 40, 2), (12, 12, 3)])
def test_lu_equals_lapack_partial_pivoting(m, l, seed):
    """LAPACK's getrf (through scipy) pivots on the first largest magnitude,
    as the oracle does: scipy returns Y = P L_s U_s, so the oracle's L (rows
    in Y's order) is P L_s and its U is U_s."""
    Y = np.random.default_rng(seed).standard_normal((m, l))
    L, U, perm = oracle.lu_pivot(Y)
    P, Ls, Us = scipy.linalg.lu(Y)
    np.testing.assert_allclose(L, P @ Ls, atol=1e-12)
    np.testing.assert_allclose(U, Us, atol=1e-12)


def test_lu_ties_go_to_the_first_row():
    """Equal magnitudes: the first row in the current order wins (integer
    entries make the ties exact)."""
    Y = np.array([[1.0, 2.0], [-3.0, 1.0], [3.0, 5.0], [2.0, -4.0]])
    L, U, perm = oracle.lu_pivot(Y)
    P, Ls, Us = scipy.linalg.lu(Y)
    assert perm[0] == 1  # |-3| and |3| tie; row 1 comes first
    np.testing.assert_allclose(L, P @ Ls, atol=1e-14)
    np.testing.assert_allclose(U, Us, atol=1e-14)


def test_lu_factors_reconstruct_and_are_bounded():
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((400, 30)) * np.exp2(rng.integers(-8, 8, size=(1, 30)))
    L, U, perm = oracle.lu_pivot(Y)
    np.testing.assert_allclose(L @ U, Y, atol=1e-13 * np.abs(Y).max())
    assert np.abs(L).max() <= 1.0 + 1e-15
    # the pivot rows of L form a unit lower triangle; U is upper triangular
    Lp = L[perm]
    np.testing.assert_array_equal(np.diag(Lp), 1.0)
    assert np.all(np.triu(Lp, 1) == 0.0)
    assert np.all(np.tril(U, -1) == 0.0)
    assert len(set(perm.tolist())) == 30
    # span(L) = span(Y)
    assert sin_theta(L, Y) < 1e-12


def test_lu_of_a_rank_deficient_matrix():
    """A column in the span of the earlier ones gives a zero pivot: U's
    diagonal entry is zero, L's column is zero below its pivot row, and Y = L U
    still holds."""
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((60, 5))
    Y[:, 3] = 2.0 * Y[:, 0] - Y[:, 2]
    L, U, perm = oracle.lu_pivot(Y)
    np.testing.assert_allclose(L @ U, Y, atol=1e-12)
    assert abs(U[3, 3]) < 1e-12


@pytest.mark.parametrize("q", [1, 2, 3])
def test_norm_iterations_match_subspace_iterations(q):
    """Every LU step keeps the span of its input, as every QR step does, so in
    exact arithmetic the two schemes give the same sketch and the same SVD; in
    FP64 on a well-conditioned problem they agree to rounding."""
    A = inputs.planted(800, 300, inputs.exp_spectrum(300, 0.05), seed=11)
    d_q, U_q, V_q = oracle.rsvd(A, 20, p=10, q=q, seed=4, scheme="qr")
    d_l, U_l, V_l = oracle.rsvd(A, 20, p=10, q=q, seed=4, scheme="lu")
    np.testing.assert_allclose(d_l, d_q, rtol=1e-10)
    assert sin_theta(U_l, U_q) < 1e-8 and sin_theta(V_l, V_q) < 1e-8
    Q, B = oracle.rqb(A, 20, p=10, q=q, seed=4, scheme="lu")
    np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
    # and the span is that of the direct power scheme (Algorithm poweriter_direct)
    Y = oracle.power_direct(A, 30, q, seed=4)
    assert sin_theta(Q, Y) < 1e-8


def test_schemes_coincide_without_iterations():
    A = inputs.planted(300, 200, inputs.exp_spectrum(200, 0.1), seed=12)
    r0 = oracle.rsvd(A, 10, p=5, q=0, seed=2, scheme="qr")
    r1 = oracle.rsvd(A, 10, p=5, q=0, seed=2, scheme="lu")
    for a, b in zip(r0, r1):
        np.testing.assert_array_equal(a, b)
