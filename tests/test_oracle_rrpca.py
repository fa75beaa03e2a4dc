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
