"""Pins of the FP64 oracle's randomized PCA (Algorithm rpca, Sec. 4.2, with
the centring / scaling of the rpca() interface, Sec. 4.4) against facts fixed
by the mathematics and by library routines -- never against the oracle's own
formulas.

With l = min(m, n) the randomized SVD is exact, so rpca must reproduce the
textbook PCA: the eigen-decomposition of the sample correlation (or
covariance) matrix computed by numpy.  Λ = Σ² / (m - 1) and Z = U Σ = X W
(Sec. 4.2) are checked through those library results.
"""
import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs


def data(m, n, rank=4, seed=3, **kw):
    return inputs.pca_data(m, n, rank, seed=seed, **kw).numpy()


def eig_desc(C):
    w, E = np.linalg.eigh(C)
    return w[::-1], E[:, ::-1]


def abs_cos(W, E):
    """|W^T E| for unit columns: 1 on the diagonal when the columns agree up to sign."""
    return np.abs(np.sum(W * E, axis=0))


@pytest.mark.parametrize("m,n,k", [(80, 12, 5), (200, 30, 8)])
def test_correlation_pca_is_exact_at_full_width(m, n, k):
    """center + scale: Λ and W are the eigenpairs of numpy's correlation
    matrix (np.corrcoef) when the sketch spans the whole row space."""
    A = data(m, n)
    r = oracle.rpca(A, k, center=True, scale=True, p=n, q=1, seed=11)
    w, E = eig_desc(np.corrcoef(A.astype(np.float64).T))
    np.testing.assert_allclose(r["eigvals"], w[:k], rtol=1e-10, atol=1e-12 * w[0])
    np.testing.assert_allclose(r["sdev"], np.sqrt(w[:k]), rtol=1e-10)
    np.testing.assert_allclose(abs_cos(r["rotation"], E[:, :k]), 1.0, atol=1e-8)
    # the trace of a correlation matrix is n: all components together explain it
    r_all = oracle.rpca(A, n - 1, center=True, scale=True, p=n, q=0, seed=11)
    assert abs(np.sum(r_all["eigvals"]) + w[-1] - n) < 1e-9 * n


def test_covariance_pca_without_scaling():
    """center only: the eigenpairs of np.cov (m - 1 denominator)."""
    A = data(150, 20)
    k = 6
    r = oracle.rpca(A, k, center=True, scale=False, p=20, q=1, seed=5)
    w, E = eig_desc(np.cov(A.astype(np.float64).T))
    np.testing.assert_allclose(r["eigvals"], w[:k], rtol=1e-10, atol=1e-12 * w[0])
    np.testing.assert_allclose(abs_cos(r["rotation"], E[:, :k]), 1.0, atol=1e-8)
    np.testing.assert_allclose(r["scale"], 1.0)


def test_no_preprocessing_is_the_svd_of_a():
    """Neither centring nor scaling: Λ (m - 1) are the squared singular values
    of A itself (numpy SVD)."""
    A = data(120, 16)
    k = 5
    r = oracle.rpca(A, k, center=False, scale=False, p=16, q=1, seed=9)
    sv = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(r["eigvals"] * (120 - 1), sv[:k] ** 2, rtol=1e-10)
    np.testing.assert_allclose(r["center"], 0.0)


def test_scaling_without_centring_uses_root_mean_square():
    """scale only: columns divided by sqrt(sum a^2 / (m - 1)), then the SVD of
    the scaled matrix (numpy)."""
    A = data(100, 10)
    k = 4
    r = oracle.rpca(A, k, center=False, scale=True, p=10, q=1, seed=2)
    Av = A.astype(np.float64)
    rms = np.sqrt(np.einsum("ij,ij->j", Av, Av) / 99.0)
    np.testing.assert_allclose(r["scale"], rms, rtol=1e-13)
    sv = np.linalg.svd(Av / rms[None, :], compute_uv=False)
    np.testing.assert_allclose(r["eigvals"], sv[:k] ** 2 / 99.0, rtol=1e-10)


def test_centre_scale_scores_and_projection():
    """center / scale outputs are numpy's mean and ddof=1 standard deviation;
    the scores Z = U Σ equal the projection X W (Sec. 4.2) and have zero
    column means."""
    A = data(300, 40)
    k = 7
    r = oracle.rpca(A, k, p=40, q=2, seed=1)  # full width: X = Q Q^T X
    Av = A.astype(np.float64)
    np.testing.assert_allclose(r["center"], Av.mean(axis=0), rtol=1e-13, atol=1e-12)
    sd = Av.std(axis=0, ddof=1)
    np.testing.assert_allclose(r["scale"], sd, rtol=1e-12)
    X = (Av - Av.mean(axis=0)) / sd
    Z = X @ r["rotation"]
    np.testing.assert_allclose(r["x"], Z, rtol=1e-8, atol=1e-9 * np.abs(Z).max())
    assert np.max(np.abs(r["x"].mean(axis=0))) < 1e-10 * np.abs(Z).max()
    # W has orthonormal columns
    np.testing.assert_allclose(r["rotation"].T @ r["rotation"], np.eye(k), atol=1e-12)


def test_invariant_to_units_and_offsets():
    """Correlation PCA does not depend on the units or origins of the
    variables: A diag(c) + 1 b^T gives the same components (same Omega)."""
    A = data(200, 24).astype(np.float64)
    rng = np.random.default_rng(4)
    c = np.exp(rng.uniform(-3, 3, 24))
    b = rng.standard_normal(24) * 100
    B = A * c[None, :] + b[None, :]
    r1 = oracle.rpca(A, 6, p=6, q=1, seed=8)
    r2 = oracle.rpca(B, 6, p=6, q=1, seed=8)
    np.testing.assert_allclose(r2["eigvals"], r1["eigvals"], rtol=1e-9)
    np.testing.assert_allclose(abs_cos(r2["rotation"], r1["rotation"]), 1.0, atol=1e-8)


def test_constant_column_contributes_nothing():
    """A zero-variance variable gets scale 0, a zero row in W, and the other
    components are those of the remaining variables."""
    A = data(150, 18, zero_var_cols=1)
    k = 5
    r = oracle.rpca(A, k, p=12, q=1, seed=6)  # l = 17 = rank of X: exact
    assert r["scale"][-1] == 0.0
    np.testing.assert_allclose(r["rotation"][-1], 0.0, atol=1e-12)
    w, _ = eig_desc(np.corrcoef(A[:, :-1].astype(np.float64).T))
    np.testing.assert_allclose(r["eigvals"], w[:k], rtol=1e-10)


def test_more_variables_than_observations():
    """m < n: at most m - 1 nonzero eigenvalues; they match numpy's covariance
    eigenvalues of the scaled data."""
    A = data(30, 90, rank=6)
    k = 10
    r = oracle.rpca(A, k, p=20, q=1, seed=7)
    assert r["rotation"].shape == (90, k) and r["x"].shape == (30, k)
    w, E = eig_desc(np.corrcoef(A.astype(np.float64).T))
    np.testing.assert_allclose(r["eigvals"], w[:k], rtol=1e-9, atol=1e-12 * w[0])
    np.testing.assert_allclose(abs_cos(r["rotation"], E[:, :k]), 1.0, atol=1e-7)


def test_bf16_values_promote_exactly():
    """BF16-stored data give the PCA of their exact values."""
    A = data(120, 14)
    bits = inputs.bf16_bits(A)
    r_b = oracle.rpca(bits, 4, p=4, q=1, seed=3)
    r_f = oracle.rpca(inputs.bf16_to_f32(bits), 4, p=4, q=1, seed=3)
    np.testing.assert_array_equal(r_b["eigvals"], r_f["eigvals"])
