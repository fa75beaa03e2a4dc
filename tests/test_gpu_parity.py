"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances (FP32 path): |sigma_i - sigma_i^o| <= 1e-5 sigma_1 and the largest
principal angle of U_k, V_k against the oracle's <= 1e-4, relaxed by the gap
rule 10 u32 ||A||_2 / (sigma_k - sigma_{k+1}) where the oracle's own spectrum
makes the rank-k subspace ill-conditioned; the full l-dimensional Q must match
within the same bound over the l-space gap.
"""
import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs
from tests.helpers import sigma_err, sin_theta, subspace_tol, ulp_distance_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    from paper_1608_02148_gb300 import build, rsvdgb
    build.build()
    assert torch.cuda.is_available()
    return rsvdgb


@pytest.fixture(scope="module")
def handle(rs):
    h = rs.Handle(0)
    yield h
    h.close()


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_rsvd(rs, handle, A_np, k, p=10, q=2, sdist="normal", seed=0, layout="row", dtype="f32",
               sig_tol=1e-5, nu=-1, nv=-1):
    import torch
    if dtype == "bf16":
        A_or = inputs.bf16_bits(A_np)
        A_dev = to_dev(A_or.view(np.int16)).view(torch.bfloat16)
    else:
        A_or = A_np
        A_dev = to_dev(A_np)
    m, n = A_np.shape
    d_o, U_o, V_o = oracle.rsvd(A_or, k, p=p, q=q, sdist=sdist, seed=seed)
    opts = rs.make_opts(p=p, q=q, sdist=sdist, seed=seed, layout=layout)
    if layout == "col":
        A_dev = A_dev.t().contiguous()  # row-major storage of A^T = column-major A
    d, U, V, info = rs.rsvdgb_rsvd(handle, A_dev, k, nu=nu, nv=nv, opts=opts)
    torch.cuda.synchronize()
    assert info.status == 0, info.as_dict()
    d = d.cpu().numpy()
    U = U.cpu().numpy()
    V = V.cpu().numpy()
    assert sigma_err(d, d_o) <= sig_tol, (sigma_err(d, d_o), d[:5], d_o[:5])
    assert np.all(np.diff(d) <= 1e-6 * d[0])
    # reference spectrum of B for the gap rule
    Aval = inputs.bf16_to_f32(A_or) if dtype == "bf16" else A_np
    l = oracle.sketch_width(m, n, k, p)
    _, _, _, Qo, Bo = oracle.rsvd(A_or, k, p=p, q=q, sdist=sdist, seed=seed, return_qb=True)
    sB = np.linalg.svd(Bo, compute_uv=False)
    tol = subspace_tol(sB, k, sB[0])
    nu_ = k if nu < 0 else nu
    nv_ = k if nv < 0 else nv
    if nu_ > 0:
        tol_u = subspace_tol(sB, nu_, sB[0])
        assert sin_theta(U, U_o[:, :nu_]) <= tol_u, (sin_theta(U, U_o[:, :nu_]), tol_u)
        assert np.max(np.abs(U.T @ U - np.eye(nu_))) < 1e-4
    if nv_ > 0:
        tol_v = subspace_tol(sB, nv_, sB[0])
        assert sin_theta(V, V_o[:, :nv_]) <= tol_v, (sin_theta(V, V_o[:, :nv_]), tol_v)
        assert np.max(np.abs(V.T @ V - np.eye(nv_))) < 1e-4
    # the whole l-dimensional basis Q against the oracle's (rqb runs the same
    # steps up to Q), within max(1e-4, 10 u32 kappa(B))
    if layout == "row" and m >= n:
        Q, _, info_q = rs.rsvdgb_rqb(handle, A_dev, k, opts=opts)
        torch.cuda.synchronize()
        assert info_q.status == 0
        tol_q = max(1e-4, 10 * 2.0 ** -24 * sB[0] / max(sB[-1], 1e-30))
        sq = sin_theta(Q.cpu().numpy(), Qo)
        assert sq <= tol_q, (sq, tol_q)
    # ||A||_F^2 and the error identity reported in info
    fa = oracle.fro2(A_or)
    assert abs(info.fro2_A - fa) <= 1e-5 * fa
    assert info.l == l
    return d, U, V, info, tol


def test_omega_bits_match_oracle(rs, handle):
    for sdist in ("normal", "unif", "rademacher"):
        for rows, l, seed in ((1000, 30, 0), (2003, 17, 2 ** 40 + 77), (7, 3, 5)):
            g = rs.rsvdgb_omega(handle, rows, l, seed=seed, sdist=sdist).cpu().numpy()
            o = oracle.omega(rows, l, seed, sdist)
            equal = np.mean(g.view(np.int32) == o.view(np.int32))
            assert equal >= 0.99999 or (rows * l < 1000 and equal == 1.0), (sdist, equal)
            assert ulp_distance_f32(g, o).max() <= 1


@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1000, 77, 1), (517, 333, 24), (260, 130, 110), (64, 640, 8)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_passes_match_oracle_products(rs, handle, m, n, l, dtype):
    import torch
    rng = np.random.default_rng(m + n + l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    X = rng.standard_normal((n, l)).astype(np.float32)
    W = rng.standard_normal((m, l)).astype(np.float32)
    if dtype == "bf16":
        Ab = inputs.bf16_bits(A)
        A_dev = to_dev(Ab.view(np.int16)).view(torch.bfloat16)
        A_or = Ab
    else:
        A_dev = to_dev(A)
        A_or = A
    Y = rs.rsvdgb_pass_ax(handle, A_dev, to_dev(X), engine="simt").cpu().numpy()
    Z = rs.rsvdgb_pass_atx(handle, A_dev, to_dev(W), engine="simt").cpu().numpy()
    Yo = oracle.gemm_ax(A_or, X.astype(np.float64))
    Zo = oracle.gemm_atx(A_or, W.astype(np.float64))
    # FP32 accumulation: error <= c K u32 sum |a||x| (deterministic bound)
    Aabs = np.abs(inputs.bf16_to_f32(A_or) if dtype == "bf16" else A).astype(np.float64)
    bound_y = 2 * n * 2 ** -24 * (Aabs @ np.abs(X)) + 1e-30
    bound_z = 2 * m * 2 ** -24 * (Aabs.T @ np.abs(W)) + 1e-30
    assert np.all(np.abs(Y - Yo) <= bound_y)
    assert np.all(np.abs(Z - Zo) <= bound_z)


def test_rsvd_small_planted_2000x1000(rs, handle):
    """2000 x 1000, sigma_i = exp(-i/20), k=20, p=10, q=2 (FP32, vs oracle)."""
    A = inputs.small_planted()
    check_rsvd(rs, handle, A, 20, p=10, q=2, seed=0)


@pytest.mark.parametrize("m,n,k,p,q", [
    (1000, 300, 10, 5, 0), (777, 333, 20, 4, 1), (300, 1000, 12, 6, 2),  # wide matrix
    (513, 257, 100, 10, 1), (256, 250, 1, 0, 1), (400, 230, 200, 20, 1),  # l = 220
    (600, 300, 170, 10, 1), (500, 260, 190, 10, 1),  # l = 180, 200: wide Jacobi and Cholesky
    (128, 64, 60, 10, 2),  # l clamps to min(m, n)
])
def test_rsvd_ragged_shapes(rs, handle, m, n, k, p, q):
    sigma = inputs.exp_spectrum(min(m, n), 3.0 / min(m, n))
    A = inputs.planted(m, n, sigma, seed=m * 7 + n)
    check_rsvd(rs, handle, A, k, p=p, q=q, seed=m)


def test_rsvd_bf16_input(rs, handle):
    A = inputs.planted(900, 400, inputs.exp_spectrum(400, 0.05), seed=3)
    check_rsvd(rs, handle, A, 16, p=8, q=1, dtype="bf16")


@pytest.mark.parametrize("shape", [(600, 250), (250, 600)])
def test_rsvd_column_major_layout(rs, handle, shape):
    A = inputs.planted(*shape, inputs.exp_spectrum(min(shape), 0.05), seed=4)
    check_rsvd(rs, handle, A, 12, p=6, q=1, layout="col")


@pytest.mark.parametrize("sdist", ["unif", "rademacher"])
def test_rsvd_other_test_matrices(rs, handle, sdist):
    A = inputs.planted(700, 300, inputs.exp_spectrum(300, 0.05), seed=5)
    check_rsvd(rs, handle, A, 15, p=10, q=1, sdist=sdist, seed=9)


def test_rsvd_nu_nv(rs, handle):
    A = inputs.planted(500, 200, inputs.exp_spectrum(200, 0.05), seed=6)
    check_rsvd(rs, handle, A, 10, p=5, q=1, nu=3, nv=0)


def test_exact_rank_gpu(rs, handle):
    """Planted rank 25 <= l = 30: sigma_1..25 to 1e-6 relative in FP32."""
    sigma = inputs.exp_spectrum(25, 1.0 / 20.0)
    A = inputs.planted(2000, 1000, sigma, seed=11)
    d, U, V, info = rs.rsvdgb_rsvd(handle, to_dev(A), 25, opts=rs.make_opts(p=5, q=0))
    d = d.cpu().numpy()
    assert info.status == 0
    assert np.max(np.abs(d - sigma) / sigma) < 1e-6, np.max(np.abs(d - sigma) / sigma)


def test_rqb_q_orthonormal_and_b_projection(rs, handle):
    A = inputs.planted(3000, 500, inputs.exp_spectrum(500, 0.02), seed=8)
    Q, B, info = rs.rsvdgb_rqb(handle, to_dev(A), 30, opts=rs.make_opts(p=10, q=2))
    Q = Q.cpu().numpy().astype(np.float64)
    B = B.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-5
    assert np.max(np.abs(B - Q.T @ A.astype(np.float64))) < 1e-5 * np.abs(A).max() * 10
    Qo, Bo = oracle.rqb(A, 30, p=10, q=2)
    sB = np.linalg.svd(Bo, compute_uv=False)
    assert sin_theta(Q, Qo) <= max(1e-4, 10 * 2 ** -24 * sB[0] / max(sB[-1], 1e-30))


@pytest.mark.parametrize("m,n,k", [(3000, 500, 30), (5000, 700, 150)])  # direct tensor-core Gram; l_pad > 128
def test_info_orth_max_is_the_basis_orthogonality(rs, handle, m, n, k):
    """opts.check_orth: info.orth_max = max |(Q^T Q - I)_ij| of the final basis
    from one FP32 Gram on the device, against the same maximum taken in FP64
    from the returned Q (the two differ by the Gram's FP32 rounding, a few
    u32); without the flag the field reads -1."""
    A = inputs.planted(m, n, inputs.exp_spectrum(n, 0.02), seed=m + k)
    Q, _, info = rs.rsvdgb_rqb(handle, to_dev(A), k, opts=rs.make_opts(p=10, q=2, check_orth=True))
    assert info.status == 0
    Q = Q.cpu().numpy().astype(np.float64)
    want = np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1])))
    assert 0.0 <= info.orth_max and abs(info.orth_max - want) <= 4e-6, (info.orth_max, want)
    d, U, V, info2 = rs.rsvdgb_rsvd(handle, to_dev(A), k, opts=rs.make_opts(p=10, q=2, check_orth=True))
    assert info2.status == 0 and abs(info2.orth_max - info.orth_max) <= 1e-6
    _, _, _, info3 = rs.rsvdgb_rsvd(handle, to_dev(A), k, opts=rs.make_opts(p=10, q=2))
    assert info3.orth_max == -1.0
    np.testing.assert_array_equal(d.cpu().numpy(), rs.rsvdgb_rsvd(handle, to_dev(A), k)[0].cpu().numpy())


def test_host_entry_point_matches_device(rs, handle):
    import torch
    A = inputs.planted(800, 300, inputs.exp_spectrum(300, 0.05), seed=12)
    d1, U1, V1, _ = rs.rsvdgb_rsvd(handle, to_dev(A), 10)
    d2, U2, V2, info = rs.rsvdgb_rsvd_host(handle, torch.from_numpy(A).pin_memory(), 10)
    assert info.status == 0
    assert np.array_equal(d1.cpu().numpy(), d2.numpy())
    assert np.array_equal(U1.cpu().numpy(), U2.numpy())


def test_invalid_arguments_rejected(rs, handle):
    import torch
    A = torch.zeros(50, 40, device="cuda")
    for k in (0, 40, 100):
        with pytest.raises(rs.RsvdgbError) as e:
            rs.rsvdgb_rsvd(handle, A, k)
        assert e.value.status == 1
    with pytest.raises(rs.RsvdgbError):
        rs.rsvdgb_rsvd(handle, A, 5, nu=6)


def test_nonfinite_input_reported(rs, handle):
    import torch
    A = torch.randn(300, 100, device="cuda")
    A[7, 3] = float("nan")
    d, U, V, info = rs.rsvdgb_rsvd(handle, A, 5, opts=rs.make_opts(q=0))
    assert info.status in (4, 5)
