"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics -- never against the oracle itself or against the CUDA path.

Each test names the passage it follows.  A plausible mistake anywhere in the
oracle (a dropped term, a wrong sign or index, a transposed operand, a wrong
rotation, a wrong Box-Muller pairing) breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1608_02148_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def sin_theta(A, B):
    """Largest principal angle sine between the column spans of A and B."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))


# --------------------------------------------------------------------------
# Test matrix (Sec. 2.3)
# --------------------------------------------------------------------------

def test_omega_gaussian_distribution():
    """Entries of the default test matrix are i.i.d. N(0,1) (Sec. 2.3)."""
    om = oracle.omega(4096, 32, seed=1234, sdist="normal").astype(np.float64)
    flat = om.ravel()
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    assert abs(flat.mean()) < 5.0 / math.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 0.02
    # columns uncorrelated
    C = np.corrcoef(om.T)
    assert np.max(np.abs(C - np.eye(32))) < 0.08


def test_omega_uniform_and_rademacher():
    """U(-1,1) and +-1 with equal probability (Sec. 2.3)."""
    u = oracle.omega(4096, 16, seed=7, sdist="unif").astype(np.float64).ravel()
    assert u.min() > -1.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    r = oracle.omega(4096, 16, seed=7, sdist="rademacher").ravel()
    assert set(np.unique(r).tolist()) == {-1.0, 1.0}
    assert abs(r.mean()) < 5.0 / math.sqrt(r.size)


def test_omega_words_feed_rows_as_specified():
    """Check the Box-Muller assembly by inverting it: for rows 4r, 4r+1 of
    column j, z0^2 + z1^2 = -2 ln u(x0) and atan2(z1, z0) = 2 pi u(x1) (mod 2 pi),
    where x0, x1 are Philox words of counter (r, 0, j, 0); likewise rows 4r+2, 4r+3
    with x2, x3.  Rademacher signs are bit 31 of x_t."""
    seed = 0x1234_5678_9ABC
    key = [seed & 0xFFFFFFFF, seed >> 32]
    om = oracle.omega(64, 8, seed, "normal").astype(np.float64)
    rad = oracle.omega(64, 8, seed, "rademacher")
    for r in (0, 3, 15):
        for j in (0, 5, 7):
            x = oracle.philox4x32_10([r, 0, j, 0], key).astype(np.float64)
            u = (x + 0.5) / 2.0 ** 32
            for h in range(2):
                z0, z1 = om[4 * r + 2 * h, j], om[4 * r + 2 * h + 1, j]
                assert abs((z0 * z0 + z1 * z1) - (-2.0 * math.log(u[2 * h]))) < 1e-5 * (1 + z0 * z0 + z1 * z1)
                ang = math.atan2(z1, z0) % (2 * math.pi)
                d = abs(ang - 2 * math.pi * u[2 * h + 1])
                assert min(d, 2 * math.pi - d) < 1e-5
            for t in range(4):
                sign = -1.0 if int(x[t]) & 0x80000000 else 1.0
                assert rad[4 * r + t, j] == sign


def test_omega_nested_columns_and_rows():
    """Columns depend only on their index, so a smaller l is a prefix (nested
    sketches); rows likewise."""
    a = oracle.omega(1001, 40, seed=99)
    b = oracle.omega(1001, 17, seed=99)
    c = oracle.omega(333, 40, seed=99)
    assert np.array_equal(a[:, :17], b)
    assert np.array_equal(a[:333], c)
    assert not np.array_equal(a, oracle.omega(1001, 40, seed=100))


def test_philox_bijective_sample_and_key_sensitivity():
    """Philox is a keyed bijection of the 128-bit counter: distinct counters
    give distinct outputs, and single-bit changes of key or counter flip about
    half of the 128 output bits (avalanche)."""
    seen = set()
    flips = []
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(2000):
        out = tuple(oracle.philox4x32_10([i, 0, 7, 0], [11, 13]).tolist())
        seen.add(out)
    assert len(seen) == 2000
    for bit in range(32):
        o2 = oracle.philox4x32_10([1 ^ (1 << bit), 2, 3, 4], [5, 6])
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, o2)))
        o3 = oracle.philox4x32_10([1, 2, 3, 4], [5 ^ (1 << bit), 6])
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, o3)))
    assert 56 < np.mean(flips) < 72


# --------------------------------------------------------------------------
# Building blocks: naive products, Householder QR, one-sided Jacobi
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_gemm_matches_library_matmul(dtype):
    rng = np.random.default_rng(3)
    full = rng.standard_normal((37, 29 + 5)).astype(np.float32)
    if dtype == "bf16":
        full_bits = inputs.bf16_bits(full)
        A = full_bits[:, :29]          # padded rows: lda = 34
        Aval = inputs.bf16_to_f32(np.ascontiguousarray(A)).astype(np.float64)
    elif dtype == "f64":
        A = full.astype(np.float64)[:, :29]
        Aval = np.ascontiguousarray(A)
    else:
        A = full[:, :29]
        Aval = np.ascontiguousarray(A).astype(np.float64)
    X = rng.standard_normal((29, 6))
    W = rng.standard_normal((37, 6))
    assert np.allclose(oracle.gemm_ax(A, X), Aval @ X, rtol=1e-13, atol=1e-12)
    assert np.allclose(oracle.gemm_atx(A, W), Aval.T @ W, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("shape", [(50, 1), (50, 7), (64, 64), (300, 40), (9, 9)])
def test_householder_qr(shape):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    Y = rng.standard_normal(shape)
    Q, R = oracle.householder_qr(Y)
    l = shape[1]
    assert np.max(np.abs(Q.T @ Q - np.eye(l))) < 1e-14 * max(1, l)
    assert np.linalg.norm(Q @ R - Y) <= 1e-14 * np.linalg.norm(Y) * max(1, l)
    assert np.allclose(np.tril(R, -1), 0.0)
    # |diag R| is unique for full-rank Y: compare with LAPACK
    _, R2 = np.linalg.qr(Y)
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(R2)), rtol=1e-12)


def test_householder_qr_rank_deficient_column():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((30, 5))
    Y[:, 2] = 0.0
    Q, R = oracle.householder_qr(Y)
    assert np.linalg.norm(Q @ R - Y) < 1e-13
    assert abs(R[2, 2]) < 1e-14


@pytest.mark.parametrize("shape", [(40, 30), (64, 64), (25, 1), (110, 110), (200, 17)])
def test_jacobi_svd_brute_force(shape):
    """Tiny inputs: the one-sided Jacobi SVD equals LAPACK's SVD."""
    rng = np.random.default_rng(shape[0] + 7 * shape[1])
    M = rng.standard_normal(shape)
    Uc, s, J, sweeps = oracle.jacobi_svd(M)
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert np.allclose(s, s_ref, rtol=1e-13, atol=1e-13 * s_ref[0])
    assert np.all(np.diff(s) <= 0)
    assert np.linalg.norm(Uc @ np.diag(s) @ J.T - M) < 1e-13 * np.linalg.norm(M)
    assert np.max(np.abs(J.T @ J - np.eye(shape[1]))) < 1e-13
    assert np.max(np.abs(Uc.T @ Uc - np.eye(shape[1]))) < 1e-12
    assert sweeps < 30


def test_jacobi_svd_rank_deficient_and_repeated():
    rng = np.random.default_rng(11)
    U, _ = np.linalg.qr(rng.standard_normal((50, 6)))
    V, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    s_true = np.array([3.0, 3.0, 1.0, 1e-3, 0.0, 0.0])
    M = U @ np.diag(s_true) @ V.T
    Uc, s, J, _ = oracle.jacobi_svd(M)
    assert np.allclose(s, s_true, atol=1e-13)
    assert np.linalg.norm(Uc @ np.diag(s) @ J.T - M) < 1e-13


# --------------------------------------------------------------------------
# Randomized SVD (Algorithms rqb, sub_iterations, rSVD)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,k,p", [((60, 40), 20, 20), ((40, 60), 20, 25), ((64, 64), 30, 34)])
def test_rsvd_with_full_width_equals_svd(shape, k, p):
    """With l = min(m, n) the sketch spans col(A) exactly, so the rSVD is the
    full SVD (Sec. 3.3 with Stage A exact)."""
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    d, U, V = oracle.rsvd(A, k, p=p, q=1, seed=3)
    Ur, sr, Vtr = np.linalg.svd(A)
    assert np.allclose(d, sr[:k], rtol=1e-12, atol=1e-12 * sr[0])
    # singular vectors up to sign (the spectrum of a Gaussian matrix is simple)
    Uc, Vc = oracle.canonical_signs(U, V)
    Urc, Vrc = oracle.canonical_signs(Ur[:, :k], Vtr.T[:, :k])
    assert np.allclose(Uc, Urc, atol=1e-9)
    assert np.allclose(Vc, Vrc, atol=1e-9)


def test_exact_rank_recovers_sigma_to_1e12():
    """Planted rank r <= l: sigma_1..sigma_r are exact to 1e-12 (Stage A
    captures col(A) when l >= rank)."""
    sigma = inputs.exp_spectrum(25, 1.0 / 20.0)
    A = inputs.planted(400, 200, sigma, seed=21, dtype=np.float64)
    d, U, V = oracle.rsvd(A, 25, p=5, q=0, seed=4)
    assert np.max(np.abs(d - sigma) / sigma) < 1e-12
    res = oracle.residual_fro2(A, U, d, V)
    assert res < 1e-24 * float(np.sum(sigma ** 2)) * 1e4


def test_rsvd_outputs_orthonormal():
    A = inputs.planted(300, 120, inputs.exp_spectrum(120, 0.05), seed=2, dtype=np.float64)
    d, U, V, Q, B = oracle.rsvd(A, 20, p=10, q=2, seed=9, return_qb=True)
    assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-13
    assert np.max(np.abs(U.T @ U - np.eye(20))) < 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(20))) < 1e-13
    assert np.all(np.diff(d) <= 0) and np.all(d > 0)
    # B = Q^T A (Eq. BQA)
    assert np.allclose(B, Q.T @ A, atol=1e-13)


def test_eckart_young_and_q_trend():
    """Eckart-Young (Sec. 3.2): no rank-k approximation beats
    sqrt(sum_{j>k} sigma_j^2); the rSVD error approaches it as q grows, the
    trend of Table tiger2 (Sec. 3.7)."""
    gold = json.load(open(GOLDEN))["tiger_table_context"]["rsvd_rel_err_by_q"]
    assert gold["0"] > gold["1"] > gold["2"] >= gold["3"]
    sigma = inputs.exp_spectrum(200, 0.02)
    A = inputs.planted(500, 200, sigma, seed=5, dtype=np.float64)
    k = 20
    opt = math.sqrt(float(np.sum(sigma[k:] ** 2)))
    errs = []
    for q in range(4):
        tot = 0.0
        for s in range(5):
            d, U, V = oracle.rsvd(A, k, p=5, q=q, seed=100 + s)
            e = math.sqrt(oracle.residual_fro2(A, U, d, V))
            assert e >= opt * (1 - 1e-12)
            tot += e
        errs.append(tot / 5)
    assert errs[0] > errs[1] > errs[2] >= errs[3] * (1 - 1e-9)
    assert errs[2] < 1.05 * opt


def hmt_bound(m, n, k, p, q, sigma_k1):
    """Right-hand side of Eq. (rsvd_expected_error), Sec. 3.4."""
    f = 1 + math.sqrt(k / (p - 1)) + math.e * math.sqrt(k + p) / p * math.sqrt(min(m, n) - k)
    return f ** (1.0 / (2 * q + 1)) * sigma_k1


@pytest.mark.parametrize("q", [0, 1])
def test_expected_error_bound(q):
    """Eq. (rsvd_expected_error) on the rank-l error ||A - QB||_2 (reading:
    the bound is stated for the full QB factorisation), averaged over 50 seeds,
    plus a Markov check: at most 10% of runs exceed 10x the bound."""
    m, n, k, p = 200, 100, 10, 5
    sigma = inputs.exp_spectrum(100, 0.08)
    A = inputs.planted(m, n, sigma, seed=31, dtype=np.float64)
    bound = hmt_bound(m, n, k, p, q, sigma[k])
    errs = []
    for s in range(50):
        Q, B = oracle.rqb(A, k, p=p, q=q, seed=1000 + s)
        errs.append(np.linalg.norm(A - Q @ B, 2))
    errs = np.array(errs)
    assert errs.mean() <= bound
    assert np.mean(errs > 10 * bound) <= 0.1
    assert errs.min() >= sigma[k + p] * (1 - 1e-9)  # cannot beat the rank-l optimum


def test_power_identity_sigma_2q_plus_1():
    """(A A^T)^q A = U Sigma^{2q+1} V^T (Sec. 2.2.2) on a 50 x 50 rank-30 matrix,
    built with the oracle's naive products and checked through its Jacobi SVD."""
    sigma = np.linspace(1.5, 0.5, 30)
    A = inputs.planted(50, 50, sigma, seed=8, dtype=np.float64)
    I = np.eye(50)
    for q in (1, 2, 3):
        M = A.copy()
        for _ in range(q):
            At_M = oracle.gemm_atx(A, M)      # A^T M
            M = oracle.gemm_ax(A, At_M)       # A A^T M
        _, s, _, _ = oracle.jacobi_svd(M)
        assert np.allclose(s[:30], sigma ** (2 * q + 1), rtol=1e-11)
        assert np.all(s[30:] < 1e-10)
    del I


def test_subspace_iteration_spans_direct_power_scheme():
    """Algorithm sub_iterations and Algorithm poweriter_direct span the same
    space in exact arithmetic; on a well-conditioned tiny case they agree."""
    sigma = np.linspace(2.0, 0.5, 40)
    A = inputs.planted(80, 40, sigma, seed=12, dtype=np.float64)
    for q in (0, 1, 2):
        Q, _ = oracle.rqb(A, 8, p=4, q=q, seed=77)
        Y = oracle.power_direct(A, 12, q, seed=77)
        assert sin_theta(Q, Y) < 1e-10


def test_error_identities():
    """Pythagorean identities used for the cheap error estimate:
    ||A - QQ^T A||_F^2 = ||A||_F^2 - ||Q^T A||_F^2 and
    ||A - U_k S_k V_k^T||_F^2 = ||A||_F^2 - sum_{i<=k} s_i^2."""
    A = inputs.planted(150, 90, inputs.exp_spectrum(90, 0.03), seed=3, dtype=np.float64)
    d, U, V, Q, B = oracle.rsvd(A, 15, p=10, q=1, seed=1, return_qb=True)
    fa = oracle.fro2(A)
    assert abs(fa - np.sum(A * A)) < 1e-12 * fa
    lhs = np.linalg.norm(A - Q @ B) ** 2
    assert abs(lhs - (fa - np.sum(B * B))) < 1e-10 * fa
    res = oracle.residual_fro2(A, U, d, V)
    assert abs(res - np.linalg.norm(A - (U * d) @ V.T) ** 2) < 1e-12 * fa
    assert abs(res - (fa - np.sum(d ** 2))) < 1e-10 * fa


def test_invariances():
    """rsvd(cA) = c rsvd(A); a row permutation of A permutes the rows of U."""
    A = inputs.planted(120, 60, inputs.exp_spectrum(60, 0.1), seed=4, dtype=np.float64)
    d, U, V = oracle.rsvd(A, 10, p=6, q=1, seed=2)
    d2, U2, V2 = oracle.rsvd(3.5 * A, 10, p=6, q=1, seed=2)
    assert np.allclose(d2, 3.5 * d, rtol=1e-12)
    Uc, Vc = oracle.canonical_signs(U, V)
    U2c, V2c = oracle.canonical_signs(U2, V2)
    assert np.allclose(Uc, U2c, atol=1e-10) and np.allclose(Vc, V2c, atol=1e-10)
    perm = np.random.default_rng(0).permutation(120)
    d3, U3, V3 = oracle.rsvd(np.ascontiguousarray(A[perm]), 10, p=6, q=1, seed=2)
    assert np.allclose(d3, d, rtol=1e-12)
    U3c, V3c = oracle.canonical_signs(U3, V3)
    assert np.allclose(U3c, Uc[perm], atol=1e-10)


@pytest.mark.parametrize("m,n", [(50, 130), (59, 60)])
def test_wide_matrix_is_transpose_problem(m, n):
    """m < n: the method factors A^T and swaps U and V (Sec. 3.3, m >= n
    without loss of generality); one column more than rows is already wide."""
    A = inputs.planted(m, n, inputs.exp_spectrum(m, 0.1), seed=6, dtype=np.float64)
    d, U, V = oracle.rsvd(A, 8, p=5, q=1, seed=3)
    dt, Ut, Vt = oracle.rsvd(np.ascontiguousarray(A.T), 8, p=5, q=1, seed=3)
    assert np.allclose(d, dt, rtol=1e-13)
    assert np.allclose(np.abs(U), np.abs(Vt), atol=1e-12)
    assert np.allclose(np.abs(V), np.abs(Ut), atol=1e-12)
    assert U.shape == (m, 8) and V.shape == (n, 8)


def test_sign_canonicalisation_convention():
    """Each pair (u_i, v_i) is flipped so that the entry of v_i of largest
    magnitude is positive (the comparison convention for singular vectors)."""
    U = np.array([[1.0, 2.0], [3.0, 4.0]])
    V = np.array([[0.1, 0.9], [-0.8, 0.2], [0.3, -0.3]])
    Uc, Vc = oracle.canonical_signs(U, V)
    np.testing.assert_array_equal(Vc, [[-0.1, 0.9], [0.8, 0.2], [-0.3, -0.3]])
    np.testing.assert_array_equal(Uc, [[-1.0, 2.0], [-3.0, 4.0]])


def test_bf16_storage_is_exact_promotion():
    """BF16-stored A gives exactly the result of its float32 promotion."""
    A32 = inputs.planted(90, 40, inputs.exp_spectrum(40, 0.1), seed=9)
    bits = inputs.bf16_bits(A32)
    d1, U1, V1 = oracle.rsvd(bits, 6, p=4, q=1, seed=5)
    d2, U2, V2 = oracle.rsvd(inputs.bf16_to_f32(bits), 6, p=4, q=1, seed=5)
    assert np.array_equal(d1, d2) and np.array_equal(U1, U2) and np.array_equal(V1, V2)


def test_padded_leading_dimension():
    A = inputs.planted(70, 30, inputs.exp_spectrum(30, 0.1), seed=1)
    padded = np.zeros((70, 37), dtype=np.float32)
    padded[:, :30] = A
    d1, U1, V1 = oracle.rsvd(A, 5, p=5, q=1, seed=8)
    d2, U2, V2 = oracle.rsvd(padded[:, :30], 5, p=5, q=1, seed=8)
    assert np.array_equal(d1, d2) and np.array_equal(U1, U2)


def test_sketch_width_clamp():
    assert oracle.sketch_width(100, 50, 10, 10) == 20
    assert oracle.sketch_width(100, 50, 45, 10) == 50
    assert oracle.sketch_width(30, 100, 25, 10) == 30


def test_paper_defaults_fixture():
    g = json.load(open(GOLDEN))
    assert g["rsvd_defaults"]["p"] == 10 and g["rsvd_defaults"]["q"] == 2
    assert g["expected_error_bound"]["requires_p_at_least"] == 2
