"""Pins of the FP64 oracle's pivoted QR, interpolative decomposition (Algorithm
id), randomized ID (Algorithm rid) and randomized CUR (Algorithm rcur),
Sec. 7 -- against library routines and exact identities, never against the
oracle's own formulas.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1608_02148_gb300 import inputs


def low_rank(m, n, r, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n))


@pytest.mark.parametrize("rows,cols,k", [(30, 50, 10), (12, 200, 12), (64, 64, 40)])
def test_pqr_matches_lapack_column_pivoting(rows, cols, k):
    """Pivots and |R| of the first k steps equal LAPACK's dgeqp3 (scipy) on
    generic matrices; R(:, piv) is upper triangular."""
    X = np.random.default_rng(rows * cols).standard_normal((rows, cols))
    piv, R, chosen, best = oracle.pqr(X, k)
    _, Rs, P = sl.qr(X, pivoting=True, mode="economic")
    np.testing.assert_array_equal(piv, P[:k])
    np.testing.assert_allclose(np.abs(R[:, piv]), np.abs(Rs[:k, :k]), atol=1e-12)
    np.testing.assert_allclose(np.abs(R[:, P[k:]]), np.abs(Rs[:k, k:]), atol=1e-12)
    assert np.max(np.abs(np.tril(R[:, piv], -1))) <= 1e-12 * np.abs(R).max()
    np.testing.assert_array_equal(chosen, best)
    assert np.all(np.diff(best) <= 1e-12)  # trailing norms of the pivots never grow


def test_pqr_ties_go_to_the_lowest_index_as_in_lapack():
    """Equal trailing norms: the pivot is the lowest column index, the choice
    of LAPACK's dgeqp3 (its idamax returns the first maximum).  Columns 3, 9
    and 14 are exact copies of the column of largest norm; each later tie
    (copies of the second-largest column) goes the same way."""
    rng = np.random.default_rng(17)
    X = rng.standard_normal((25, 20))
    X[:, 3] *= 10.0
    X[:, 9] = X[:, 3]
    X[:, 14] = X[:, 3]
    X[:, 6] *= 5.0
    X[:, 11] = X[:, 6]
    piv, _, _, _ = oracle.pqr(X, 4)
    _, _, P = sl.qr(X, pivoting=True, mode="economic")
    assert piv[0] == 3 and P[0] == 3
    assert piv[1] == 6 and P[1] == 6
    assert 9 not in piv[:2] and 14 not in piv[:2] and 11 not in piv[:2]


def test_pqr_prescribed_pivots_report_residuals():
    X = np.random.default_rng(5).standard_normal((20, 40))
    piv, _, _, _ = oracle.pqr(X, 5)
    alt = piv.copy()
    alt[2] = [j for j in range(40) if j not in piv][0]
    _, _, chosen, best = oracle.pqr(X, 5, force_piv=alt)
    assert chosen[2] < best[2]
    with pytest.raises(RuntimeError):
        oracle.pqr(X, 5, force_piv=[0, 0, 1, 2, 3])


def test_id_is_exact_at_the_rank():
    """rank(X) = k: X = X(:, J) Z exactly, Z(:, J) = I (Algorithm id)."""
    X = low_rank(40, 120, 7, 1)
    J, Z = oracle.id_decomp(X, 7)
    np.testing.assert_allclose(X[:, J] @ Z, X, atol=1e-9 * np.abs(X).max())
    np.testing.assert_allclose(Z[:, J], np.eye(7), atol=0)


def test_id_picks_the_dominant_column_first():
    X = np.random.default_rng(2).standard_normal((15, 60))
    X[:, 37] *= 100.0
    J, _ = oracle.id_decomp(X, 3)
    assert J[0] == 37


@pytest.mark.parametrize("p,q", [(0, 0), (5, 1), (10, 2)])
def test_rid_is_exact_at_the_rank(p, q):
    """Algorithm rid on an exactly rank-k A: l >= k spans its range, so
    A = C Z with C = A(:, J)."""
    A = low_rank(300, 80, 9, 3)  # float64: exactly rank 9 up to rounding
    C, Z, J, B = oracle.rid(A, 9, p=p, q=q, seed=4)
    Av = A
    np.testing.assert_array_equal(C, Av[:, J])
    np.testing.assert_allclose(C @ Z, Av, atol=1e-8 * np.abs(Av).max())


def test_rcur_is_exact_at_the_rank():
    """Algorithm rcur on an exactly rank-k A: A = C U R, C and R actual
    columns and rows of A."""
    A = low_rank(250, 90, 6, 7)
    C, U, R, J, I = oracle.rcur(A, 6, p=5, q=1, seed=2)
    Av = A
    np.testing.assert_array_equal(C, Av[:, J])
    np.testing.assert_array_equal(R, Av[I, :])
    np.testing.assert_allclose(C @ U @ R, Av, atol=1e-7 * np.abs(Av).max())
    assert len(set(I.tolist())) == 6 and len(set(J.tolist())) == 6


def test_rid_error_near_optimal_on_a_planted_spectrum():
    """On A = U diag(sigma) V^T the rank-k ID error stays within a modest
    factor of the Eckart-Young optimum (the ID is not optimal, Sec. 7)."""
    sigma = inputs.exp_spectrum(60, 0.2)
    A = inputs.planted(400, 60, sigma, seed=11)
    k = 10
    C, Z, J, _ = oracle.rid(A, k, p=10, q=2, seed=1)
    err = np.linalg.norm(A.astype(np.float64) - C @ Z)
    opt = np.sqrt(np.sum(sigma[k:] ** 2))
    assert opt < err < 10 * opt


def test_rid_bf16_values_promote_exactly():
    A = low_rank(200, 50, 5, 9).astype(np.float32)
    bits = inputs.bf16_bits(A)
    C1, Z1, J1, _ = oracle.rid(bits, 5, p=5, q=1, seed=3)
    C2, Z2, J2, _ = oracle.rid(inputs.bf16_to_f32(bits), 5, p=5, q=1, seed=3)
    np.testing.assert_array_equal(J1, J2)
    np.testing.assert_array_equal(Z1, Z2)


def test_rcur_middle_factor_is_the_least_squares_fit_of_z():
    """Algorithm rcur steps 5-6: U = Z pinv(R), i.e. the minimiser of
    ||U R - Z||_F (R of full row rank), here solved by LAPACK's least squares
    (scipy) on a matrix that is not of rank k, where other choices of U (for
    instance pinv(C) A pinv(R), the best U for the given C and R) differ."""
    rng = np.random.default_rng(11)
    A = inputs.planted(200, 70, np.exp(-0.15 * np.arange(70)), seed=6, dtype=np.float64)
    A = A + 1e-3 * rng.standard_normal(A.shape)
    k = 8
    C, U, R, J, I = oracle.rcur(A, k, p=6, q=1, seed=5)
    _, Z, _, _ = oracle.rid(A, k, p=6, q=1, seed=5)
    U_ls = sl.lstsq(R.T, Z.T)[0].T
    np.testing.assert_allclose(U, U_ls, rtol=0, atol=1e-9 * np.abs(U_ls).max())
    U_best = np.linalg.pinv(C) @ A @ np.linalg.pinv(R)
    assert np.abs(U_best - U).max() > 1e-6 * np.abs(U).max()


def test_pqr_reports_two_norms_of_the_trailing_columns():
    """At step 0 the trailing part of every column is the whole column, so
    the reported largest residual is the largest column 2-norm (numpy), and
    at step 1 it is the largest norm of the columns projected off the first
    pivot."""
    X = np.random.default_rng(8).standard_normal((30, 45))
    piv, _, chosen, best = oracle.pqr(X, 3)
    norms = np.linalg.norm(X, axis=0)
    assert abs(best[0] - norms.max()) <= 1e-13 * norms.max()
    assert abs(chosen[0] - norms[piv[0]]) <= 1e-13 * norms.max()
    q0 = X[:, piv[0]] / norms[piv[0]]
    P = X - np.outer(q0, q0 @ X)
    P[:, piv[0]] = 0.0
    assert abs(best[1] - np.linalg.norm(P, axis=0).max()) <= 1e-12 * norms.max()


def test_rid_factors_the_rqb_factor_with_the_papers_p_and_q():
    """Algorithm rid step 1 is rqb(A, k, p, q) with the same p and q as
    everywhere (the listing's swapped order is read as a typo): B has
    l = k + p rows and is the B of rqb with those arguments."""
    A = inputs.planted(150, 60, inputs.exp_spectrum(60, 0.1), seed=3, dtype=np.float64)
    C, Z, J, B = oracle.rid(A, 5, p=7, q=1, seed=2)
    _, B_rqb = oracle.rqb(A, 5, p=7, q=1, seed=2)
    assert B.shape == (12, 60)
    np.testing.assert_array_equal(B, B_rqb)
