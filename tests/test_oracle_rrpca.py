"""Pins of the FP64 oracle's randomized robust PCA (Algorithm rrpca, Sec. 5,
the inexact augmented Lagrange multiplier method) against facts fixed by the
mathematics and by library routines.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs


def test_soft_threshold_and_rank_prediction():
    x = np.array([-3.0, -0.5, 0.0, 0.2, 2.0])
    np.testing.assert_array_equal(oracle.soft_threshold(x, 1.0), [-2.0, 0.0, 0.0, 0.0, 1.0])
    d = np.array([5.0, 3.0, 0.4, 0.1])
    # 2 of 4 above 1/mu = 1: fewer than the target rank 4 -> 3
    assert oracle.predict_rank(d, 1.0, 4, 100, 200) == (3, 2)
    # all above: grow by 5 % of min(m, n) = 10
    assert oracle.predict_rank(d, 0.01, 4, 100, 200) == (14, 4)
    assert oracle.predict_rank(d, 0.01, 4, 9, 200) == (9, 4)


def test_full_width_sketch_is_the_textbook_ialm():
    """With p large enough that l = min(m, n) the randomized SVD is exact, so
    the iteration must follow the same iteration run with numpy's full SVD."""
    L0, S0, A = inputs.low_rank_plus_sparse(60, 40, 3, 0.1, seed=2)

    def exact(X, k):
        U, d, Vt = np.linalg.svd(X, full_matrices=False)
        return d[:k], U[:, :k], Vt[:k].T

    r1 = oracle.rrpca(A, p=40, q=1, seed=1, maxiter=30)
    r2 = oracle.rrpca(A, p=40, q=1, seed=1, maxiter=30, svd=exact)
    assert r1["iters"] == r2["iters"]
    np.testing.assert_allclose(r1["L"], r2["L"], atol=1e-8)
    np.testing.assert_allclose(r1["S"], r2["S"], atol=1e-8)


@pytest.mark.parametrize("m,n,rank,density", [(300, 300, 5, 0.2), (400, 120, 4, 0.1)])
def test_recovers_low_rank_and_sparse_parts(m, n, rank, density):
    """Principal component pursuit recovers L0 and S0 exactly for low rank and
    sparse corruptions (the guarantee the IALM solves for); the paper's
    300 x 300 rank-5, 20 % case is the first."""
    L0, S0, A = inputs.low_rank_plus_sparse(m, n, rank, density, seed=7)
    r = oracle.rrpca(A, seed=3)
    assert r["err"] < 1e-5 and r["iters"] < 50
    assert np.linalg.norm(r["L"] - L0) < 1e-4 * np.linalg.norm(L0)
    assert np.linalg.norm(r["S"] - S0) < 1e-4 * np.linalg.norm(S0)
    assert np.linalg.matrix_rank(r["L"], tol=1e-6 * np.linalg.norm(r["L"], 2)) == rank
    assert np.linalg.norm(A - r["L"] - r["S"]) <= 1e-5 * np.linalg.norm(A)


def test_the_papers_simulation_case():
    """The simulation of Sec. 5.5 (sizes, rank, corruption range and
    fraction from tests/golden): recovery of L to the stopping tolerance
    scaled by ||A|| / ||L|| and of S to 1e-4, rank exact."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    ex = gold["rrpca_example"]
    m, n = ex["shape"]
    for seed in (1, 2):
        L0, S0, A = inputs.rrpca_example(seed, m, n, ex["rank"], ex["sparse_fraction"])
        assert np.abs(S0).max() <= ex["sparse_range"][1]
        r = oracle.rrpca(A, seed=3)
        assert r["err"] < 1e-5 and r["svp"] == ex["rank"]
        tol_L = 10 * 1e-5 * np.linalg.norm(A) / np.linalg.norm(L0)
        assert np.linalg.norm(r["L"] - L0) < tol_L * np.linalg.norm(L0)
        assert np.linalg.norm(r["S"] - S0) < 1e-4 * np.linalg.norm(S0)


def test_default_lambda_is_the_papers():
    """lambda = max(m, n)^(-1/2) by default (Sec. 5, with the rrpca()
    signature of Sec. 5.4), checked on a rectangular case where the choice
    changes the result."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    assert gold["rrpca_defaults"]["lambda"] == "max(m, n)^(-1/2)"
    L0, S0, A = inputs.low_rank_plus_sparse(160, 60, 3, 0.05, seed=4)
    m, n = A.shape
    r = oracle.rrpca(A, seed=2, maxiter=40)
    r_max = oracle.rrpca(A, lam=max(m, n) ** -0.5, seed=2, maxiter=40)
    r_min = oracle.rrpca(A, lam=min(m, n) ** -0.5, seed=2, maxiter=40)
    np.testing.assert_array_equal(r["S"], r_max["S"])
    np.testing.assert_array_equal(r["L"], r_max["L"])
    assert np.abs(r["S"] - r_min["S"]).max() > 1e-6 * np.abs(r["S"]).max()


def _dual_norm(Z, lam):
    """Norm of the dual-feasible set of principal component pursuit.  The
    Lagrangian of min ||L||_* + lam ||S||_1 s.t. A = L + S is bounded below
    in L only while ||Z||_2 <= 1 (the dual of the nuclear norm) and in S only
    while max|z_ij| <= lam (the dual of lam ||.||_1): the multiplier is feasible
    exactly when this gauge is at most 1."""
    return max(np.linalg.norm(Z, 2), np.abs(Z).max() / lam)


@pytest.mark.parametrize("case", ["spectral", "entrywise"])
def test_initial_multiplier_is_a_on_the_dual_boundary(case):
    """Algorithm rrpca step 3 scales A by the inverse of its dual norm.  A
    positive multiple of A whose gauge is exactly 1 is unique, so checking
    both properties pins Z_0 (on one matrix where the spectral term decides
    and one where a large entry does)."""
    rng = np.random.default_rng(5)
    if case == "spectral":
        A = 1.0 + 0.1 * rng.standard_normal((40, 30))  # ||A||_2 ~ 35 > max|a| / lam ~ 8
    else:
        A = rng.standard_normal((40, 30))  # max|a| / lam ~ 20 > ||A||_2 ~ 12
    lam = 1.0 / np.sqrt(40)
    Z0 = oracle.rrpca(A, maxiter=0)["Z"]
    c = Z0[np.nonzero(A)] / A[np.nonzero(A)]
    assert np.all(c > 0) and np.ptp(c) <= 1e-12 * c.max()
    assert abs(_dual_norm(Z0, lam) - 1.0) < 1e-12
    spectral = np.linalg.norm(Z0, 2) > np.abs(Z0).max() / lam
    assert spectral == (case == "spectral")


def test_first_iterate_by_hand():
    """A = diag(3, 1), lambda = 1/sqrt(2), worked by hand.
    ||A||_2 = 3 and max|a| / lambda = 3 sqrt(2), so Z_0 = A / (3 sqrt(2)) and
    mu_0 = 1.25 / 3.  X = A + Z_0 / mu_0 = c A with c = 1 + 1 / (1.25 sqrt(2)).
    The target rank starts at min(2, min(m, n) - 1) = 1 and the rank-1 factor
    of the diagonal X is exact: sigma = 3c > 1 / mu_0 = 2.4, so svp = 1 and
    L = (3c - 2.4) e1 e1^T.  A - L + Z_0 / mu_0 = diag(2.4, c) soft-thresholded
    at lambda / mu_0 = 2.4 / (1.25 sqrt(2)) gives S = diag(2.4 - 2.4 /
    (1.25 sqrt(2)), 0); the residual A - L - S = diag(0, 1), so
    Z_1 = Z_0 + mu_0 diag(0, 1) and mu_1 = 1.5 mu_0."""
    A = np.diag([3.0, 1.0])
    r = oracle.rrpca(A, maxiter=1, tol=0.0)
    s2 = np.sqrt(2.0)
    c = 1.0 + 1.0 / (1.25 * s2)
    mu0 = 1.25 / 3.0
    thr = (1.0 / s2) / mu0
    np.testing.assert_allclose(r["L"], np.diag([3 * c - 2.4, 0.0]), atol=1e-12)
    np.testing.assert_allclose(r["S"], np.diag([2.4 - thr, 0.0]), atol=1e-12)
    np.testing.assert_allclose(r["Z"], np.diag([3.0 / (3 * s2), 1.0 / (3 * s2) + mu0]), atol=1e-12)
    np.testing.assert_allclose(r["mu_hist"], [mu0, 1.5 * mu0], rtol=1e-14)
    assert r["svp"] == 1


def test_penalty_grows_geometrically_to_a_finite_cap():
    """The penalty mu grows by rho = 1.5 per iteration and stops at a cap: a
    bounded mu keeps sum 1 / mu_k divergent, the condition under which the
    inexact method converges to the optimum rather than stalling at a
    non-optimal point.  The cap's value (10^7 mu_0) is the cited method's
    choice, checked here where the iteration reaches it."""
    L0, S0, A = inputs.low_rank_plus_sparse(30, 20, 2, 0.1, seed=9)
    r = oracle.rrpca(A, maxiter=60, tol=0.0, seed=1)
    mu = np.asarray(r["mu_hist"])
    assert np.all(np.diff(mu) >= 0)
    cap = mu[-1]
    assert np.all(mu <= cap)
    np.testing.assert_allclose(cap / mu[0], 1e7, rtol=1e-12)
    first = int(np.argmax(mu >= cap))  # first iterate at the cap
    assert 0 < first < len(mu) - 1
    # strictly geometric before it, reached at the first step that would overshoot it
    np.testing.assert_allclose(mu[1:first] / mu[:first - 1], 1.5, rtol=1e-12)
    assert mu[first - 1] * 1.5 >= cap
    np.testing.assert_array_equal(mu[first:], cap)
