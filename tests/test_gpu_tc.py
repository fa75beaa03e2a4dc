"""Parity of the tensor-core (tcgen05 + TMA) passes over A with the FP64
oracle, through the C ABI, in both FP32-accurate forms.

Error model of one 3xTF32 product (engine tc_tf32): a_hi p_hi + a_hi p_lo +
a_lo p_hi with the lo parts rounded to TF32 and a_lo p_lo dropped leaves at
most 2^-20 |a||p| per product; FP32 accumulation adds K u32 |a||p|.  The
bound below is (2^-19 + 2 K u32) (|A| |X|) element by element.
Scaled FP16x3 (engine tc): A scaled by 2^eA and each panel column by 2^ej
(largest magnitude into [2^13, 2^14)), both split into FP16 hi + lo; the
same three products leave at most 2^-20 |a||p| while the lo parts are
normal FP16 numbers, and below that an absolute 2^-25 in scaled units, i.e.
2^-38 max|A| per element of A (2^-38 max|x_j| per panel element): the bound
gains K 2^-37 max|A| max|X|, which only matters for rows many orders of
magnitude below the largest.
"""
import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs
from tests.helpers import sigma_err, sin_theta, subspace_tol

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


def _product_bounds(A, X, W, engine):
    Aa = np.abs(A).astype(np.float64)
    m, n = A.shape
    by = (2.0 ** -19 + 2 * n * 2.0 ** -24) * (Aa @ np.abs(X))
    bz = (2.0 ** -19 + 2 * m * 2.0 ** -24) * (Aa.T @ np.abs(W))
    if engine == "tc":
        amax = float(Aa.max())
        by = by + n * 2.0 ** -37 * amax * np.abs(X).max(axis=0)[None, :]
        bz = bz + m * 2.0 ** -37 * amax * np.abs(W).max(axis=0)[None, :]
    return by, bz


@pytest.mark.parametrize("engine", ["tc", "tc_tf32"])
@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1000, 64, 1), (520, 332, 24), (260, 128, 110),
                                   (64, 640, 8), (1030, 516, 220), (4096, 256, 256), (777, 1000, 112)])
def test_tc_passes_match_oracle_products(rs, handle, m, n, l, engine):
    rng = np.random.default_rng(7 * m + n + l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    X = rng.standard_normal((n, l)).astype(np.float32)
    W = rng.standard_normal((m, l)).astype(np.float32)
    Ad = to_dev(A)
    Y = rs.rsvdgb_pass_ax(handle, Ad, to_dev(X), engine=engine).cpu().numpy().astype(np.float64)
    Z = rs.rsvdgb_pass_atx(handle, Ad, to_dev(W), engine=engine).cpu().numpy().astype(np.float64)
    Yo = oracle.gemm_ax(A, X.astype(np.float64))
    Zo = oracle.gemm_atx(A, W.astype(np.float64))
    by, bz = _product_bounds(A, X, W, engine)
    assert np.all(np.abs(Y - Yo) <= by), float(np.max(np.abs(Y - Yo) / by))
    assert np.all(np.abs(Z - Zo) <= bz), float(np.max(np.abs(Z - Zo) / bz))


@pytest.mark.parametrize("engine", ["tc", "tc_tf32"])
def test_tc_passes_rows_of_very_different_scale(rs, handle, engine):
    """Rows and panel columns spread over 2^-30 .. 2^10 of magnitude (and a
    zero row): the FP16x3 form keeps the relative bound for the rows near
    max|A| and the absolute floor K 2^-37 max|A| max|x_j| for the others."""
    rng = np.random.default_rng(99)
    m, n, l = 1500, 700, 40
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-30, 11, size=(m, 1)))
    A[17] = 0.0
    A = A.astype(np.float32)
    X = (rng.standard_normal((n, l)) * np.exp2(rng.integers(-20, 8, size=(1, l)))).astype(np.float32)
    W = (rng.standard_normal((m, l)) * np.exp2(rng.integers(-20, 8, size=(1, l)))).astype(np.float32)
    Ad = to_dev(A)
    Y = rs.rsvdgb_pass_ax(handle, Ad, to_dev(X), engine=engine).cpu().numpy().astype(np.float64)
    Z = rs.rsvdgb_pass_atx(handle, Ad, to_dev(W), engine=engine).cpu().numpy().astype(np.float64)
    Yo = oracle.gemm_ax(A, X.astype(np.float64))
    Zo = oracle.gemm_atx(A, W.astype(np.float64))
    by, bz = _product_bounds(A, X, W, engine)
    assert np.all(np.abs(Y - Yo) <= by), float(np.max(np.abs(Y - Yo) / by))
    assert np.all(np.abs(Z - Zo) <= bz), float(np.max(np.abs(Z - Zo) / bz))
    assert np.all(Y[17] == 0.0)


def test_tc_rejects_unaligned_rows(rs, handle):
    import torch
    A = torch.zeros(100, 33, device="cuda")  # lda = 33 floats: rows not 16-byte aligned
    X = torch.zeros(33, 8, device="cuda")
    with pytest.raises(rs.RsvdgbError) as e:
        rs.rsvdgb_pass_ax(handle, A, X, engine="tc")
    assert e.value.status == 7


@pytest.mark.parametrize("engine", ["tc", "tc_tf32"])
@pytest.mark.parametrize("m,n,k,p,q", [(2000, 1000, 20, 10, 2), (513, 256, 100, 10, 1), (300, 1000, 12, 6, 2),
                                       (400, 232, 200, 20, 1), (4096, 64, 10, 6, 3)])
def test_tc_rsvd_matches_oracle(rs, handle, m, n, k, p, q, engine):
    import torch
    sigma = inputs.exp_spectrum(min(m, n), 3.0 / min(m, n)) if (m, n) != (2000, 1000) else \
        inputs.exp_spectrum(1000, 1.0 / 20.0)
    A = inputs.planted(m, n, sigma, seed=m + 3 * n)
    d_o, U_o, V_o, Q_o, B_o = oracle.rsvd(A, k, p=p, q=q, seed=5, return_qb=True)
    d, U, V, info = rs.rsvdgb_rsvd(handle, to_dev(A), k, opts=rs.make_opts(p=p, q=q, seed=5, engine=engine))
    torch.cuda.synchronize()
    assert info.status == 0, info.as_dict()
    assert info.engine == {"tc": 2, "tc_tf32": 3}[engine]
    assert sigma_err(d.cpu().numpy(), d_o) <= 1e-5, sigma_err(d.cpu().numpy(), d_o)
    sB = np.linalg.svd(B_o, compute_uv=False)
    tol = subspace_tol(sB, k, sB[0])
    assert sin_theta(U.cpu().numpy(), U_o) <= tol
    assert sin_theta(V.cpu().numpy(), V_o) <= tol
    fa = oracle.fro2(A)
    assert abs(info.fro2_A - fa) <= 1e-5 * fa


def test_tc_and_simt_engines_agree(rs, handle):
    A = inputs.planted(3000, 400, inputs.exp_spectrum(400, 0.03), seed=77)
    Ad = to_dev(A)
    d1, U1, V1, _ = rs.rsvdgb_rsvd(handle, Ad, 30, opts=rs.make_opts(engine="tc"))
    d2, U2, V2, _ = rs.rsvdgb_rsvd(handle, Ad, 30, opts=rs.make_opts(engine="simt"))
    d1, d2 = d1.cpu().numpy(), d2.cpu().numpy()
    assert np.max(np.abs(d1 - d2)) <= 2e-5 * d2[0]


@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1030, 516, 220), (4096, 256, 100), (520, 332, 8)])
def test_bf16_passes_match_oracle_products(rs, handle, m, n, l):
    """BF16 products: both operands rounded to nearest BF16 (relative error
    <= 2^-9 each), FP32 accumulation: |Y - Y_o| <= (2^-8 + 2 K u32) |A||X|."""
    rng = np.random.default_rng(11 * m + n + l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    X = rng.standard_normal((n, l)).astype(np.float32)
    W = rng.standard_normal((m, l)).astype(np.float32)
    Ad = to_dev(A)
    Y = rs.rsvdgb_pass_ax(handle, Ad, to_dev(X), engine="tc", prec="bf16_sketch").cpu().numpy().astype(np.float64)
    Z = rs.rsvdgb_pass_atx(handle, Ad, to_dev(W), engine="tc", prec="bf16_sketch").cpu().numpy().astype(np.float64)
    Yo = oracle.gemm_ax(A, X.astype(np.float64))
    Zo = oracle.gemm_atx(A, W.astype(np.float64))
    Aa = np.abs(A).astype(np.float64)
    by = (2.0 ** -8 + 2 * n * 2.0 ** -24) * (Aa @ np.abs(X))
    bz = (2.0 ** -8 + 2 * m * 2.0 ** -24) * (Aa.T @ np.abs(W))
    assert np.all(np.abs(Y - Yo) <= by)
    assert np.all(np.abs(Z - Zo) <= bz)
    # and it is not secretly FP32-accurate: BF16 rounding is visible
    assert np.max(np.abs(Y - Yo) / by) > 1e-3


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 1000, 20, 10, 2), (3000, 512, 100, 10, 2), (800, 300, 16, 8, 1)])
def test_bf16_sketch_rsvd_equal_error(rs, handle, m, n, k, p, q):
    """Mixed precision (BF16 sketch and power passes, FP32-accurate projection):
    ||A - U S V^T||_F <= 1.01 x the oracle's at the same (k, p, q)."""
    import torch
    if (m, n) == (2000, 1000):
        A = inputs.small_planted()
    else:
        A = inputs.planted(m, n, inputs.exp_spectrum(min(m, n), 2.0 / k), seed=m + n)
    d_o, U_o, V_o = oracle.rsvd(A, k, p=p, q=q, seed=3)
    err_o = np.sqrt(oracle.residual_fro2(A, U_o, d_o, V_o))
    d, U, V, info = rs.rsvdgb_rsvd(handle, to_dev(A), k,
                                   opts=rs.make_opts(p=p, q=q, seed=3, prec="bf16_sketch"))
    torch.cuda.synchronize()
    assert info.status == 0 and info.engine == 2
    err = np.sqrt(oracle.residual_fro2(A, U.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64),
                                       V.cpu().numpy().astype(np.float64)))
    assert err <= 1.01 * err_o, (err, err_o)
    # the device's own estimate of the rank-k error agrees with the explicit residual
    assert abs(np.sqrt(max(info.err2_k, 0.0)) - err) <= 1e-3 * np.sqrt(oracle.fro2(A)) + 1e-3 * err


@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1030, 520, 220), (4096, 256, 100), (777, 1000, 112), (64, 640, 8)])
@pytest.mark.parametrize("prec", ["fp32", "bf16_sketch"])
def test_tc_passes_bf16_stored_a(rs, handle, m, n, l, prec):
    """A stored in BF16 (Sec. 3.6 allows any numeric matrix; the C3 workload
    stores A in BF16).  BF16 values are exact in TF32, so the FP32-accurate
    product needs a p_hi + a p_lo only and meets the same bound,
    (2^-19 + 2 K u32)(|A||X|); in mixed precision the BF16 panel bound holds."""
    import torch
    rng = np.random.default_rng(5 * m + n + l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    Ab = inputs.bf16_bits(A)
    Aval = inputs.bf16_to_f32(Ab).astype(np.float64)
    A_dev = to_dev(Ab.view(np.int16)).view(torch.bfloat16)
    X = rng.standard_normal((n, l)).astype(np.float32)
    W = rng.standard_normal((m, l)).astype(np.float32)
    Y = rs.rsvdgb_pass_ax(handle, A_dev, to_dev(X), engine="tc", prec=prec).cpu().numpy().astype(np.float64)
    Z = rs.rsvdgb_pass_atx(handle, A_dev, to_dev(W), engine="tc", prec=prec).cpu().numpy().astype(np.float64)
    Yo = oracle.gemm_ax(Ab, X.astype(np.float64))
    Zo = oracle.gemm_atx(Ab, W.astype(np.float64))
    c = 2.0 ** -19 if prec == "fp32" else 2.0 ** -8
    by = (c + 2 * n * 2.0 ** -24) * (np.abs(Aval) @ np.abs(X))
    bz = (c + 2 * m * 2.0 ** -24) * (np.abs(Aval).T @ np.abs(W))
    assert np.all(np.abs(Y - Yo) <= by), float(np.max(np.abs(Y - Yo) / by))
    assert np.all(np.abs(Z - Zo) <= bz), float(np.max(np.abs(Z - Zo) / bz))


@pytest.mark.parametrize("prec", ["fp32", "bf16_sketch"])
def test_tc_rsvd_bf16_stored_a(rs, handle, prec):
    """rSVD of a BF16-stored A on the tensor cores against the oracle run on
    the same BF16 values: FP32 tolerances for the FP32 path, equal error
    (<= 1.01 x the oracle's) for the mixed one."""
    import torch
    A = inputs.planted(3000, 512, inputs.exp_spectrum(512, 0.04), seed=31)
    Ab = inputs.bf16_bits(A)
    A_dev = to_dev(Ab.view(np.int16)).view(torch.bfloat16)
    k = 40
    d_o, U_o, V_o, Q_o, B_o = oracle.rsvd(Ab, k, p=10, q=2, seed=8, return_qb=True)
    d, U, V, info = rs.rsvdgb_rsvd(handle, A_dev, k, opts=rs.make_opts(p=10, q=2, seed=8, prec=prec))
    torch.cuda.synchronize()
    assert info.status == 0 and info.engine == 2
    if prec == "fp32":
        assert sigma_err(d.cpu().numpy(), d_o) <= 1e-5
        sB = np.linalg.svd(B_o, compute_uv=False)
        tol = subspace_tol(sB, k, sB[0])
        assert sin_theta(U.cpu().numpy(), U_o) <= tol
        assert sin_theta(V.cpu().numpy(), V_o) <= tol
    else:
        Aval = inputs.bf16_to_f32(Ab).astype(np.float64)
        err_o = np.sqrt(oracle.residual_fro2(Aval, U_o, d_o, V_o))
        err = np.sqrt(oracle.residual_fro2(Aval, U.cpu().numpy().astype(np.float64),
                                           d.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)))
        assert err <= 1.01 * err_o, (err, err_o)


def test_full_size_scale_of_products(rs, handle):
    """200000 x 2000 (the benchmark's size): the tensor core's FP32
    accumulation truncates, which would shrink long sums; the products whose
    scale matters are accumulated in short chunks.  Against FP64 products of
    the same stored values: the relative scale error of A^T X and of the
    projection B = Q^T A stays below 5e-6, and Q from CholeskyQR2 (Grams of
    200000 rows) is orthonormal to 2e-6 on its diagonal."""
    import torch
    m, n = 200000, 2000
    A = inputs.spiked_noise(m, n, 1.0 / np.arange(1, n + 1), 1e-3, seed=0x160802148 + 2000, device="cuda")
    A64 = A.double()

    def scale_err(X, X64):
        X = X.double()
        return float((X * X64).sum() / (X64 * X64).sum() - 1.0)

    Xm = torch.randn(m, 110, device="cuda")
    Z = rs.rsvdgb_pass_atx(handle, A, Xm)
    assert abs(scale_err(Z, A64.T @ Xm.double())) < 5e-6
    Q, B, info = rs.rsvdgb_rqb(handle, A, 100, rs.make_opts(p=10, q=2))
    torch.cuda.synchronize()
    assert info.status == 0
    Q64 = Q.double()
    d = torch.diagonal(Q64.T @ Q64)
    assert float(torch.max(torch.abs(d - 1))) < 2e-6
    assert abs(scale_err(B, Q64.T @ A64)) < 5e-6


@pytest.mark.parametrize("m,n,l", [(300, 200, 30), (1030, 520, 220), (4096, 256, 100), (777, 1024, 112), (64, 640, 8),
                                   (200, 2104, 40), (90, 4200, 24)])
@pytest.mark.parametrize("stored", ["f32", "bf16"])
def test_fp8_passes_match_oracle_products(rs, handle, m, n, l, stored):
    """E4M3 products: A's rows and the panel's columns scaled by powers of two
    into E4M3's range and rounded to nearest (relative error <= 2^-4 each in
    the normal range), FP32 accumulation: |Y - Y_o| <= (2^-3 + 2^-7 + 2 K u32)
    |A||X| plus K 2^-18 max_i|a| max_j|x| for entries below E4M3's normal
    range; and visibly not BF16-accurate.  n > 2048 takes the prep kernel's
    two-read path (rows wider than a register-resident chunk)."""
    import torch
    rng = np.random.default_rng(3 * m + n + l)
    A = (rng.standard_normal((m, n)) * np.exp2(rng.integers(-6, 6, size=(m, 1)))).astype(np.float32)
    if stored == "bf16":
        Ab = inputs.bf16_bits(A)
        A_dev = to_dev(Ab.view(np.int16)).view(torch.bfloat16)
        A_or = Ab
        Aval = inputs.bf16_to_f32(Ab).astype(np.float64)
    else:
        A_dev = to_dev(A)
        A_or = A
        Aval = A.astype(np.float64)
    X = rng.standard_normal((n, l)).astype(np.float32)
    W = rng.standard_normal((m, l)).astype(np.float32)
    Y = rs.rsvdgb_pass_ax(handle, A_dev, to_dev(X), engine="tc", prec="fp8_sketch").cpu().numpy().astype(np.float64)
    Z = rs.rsvdgb_pass_atx(handle, A_dev, to_dev(W), engine="tc", prec="fp8_sketch").cpu().numpy().astype(np.float64)
    Yo = oracle.gemm_ax(A_or, X.astype(np.float64))
    Zo = oracle.gemm_atx(A_or, W.astype(np.float64))
    Aa = np.abs(Aval)
    c = 2.0 ** -3 + 2.0 ** -7
    by = (c + 2 * n * 2.0 ** -24) * (Aa @ np.abs(X)) + n * 2.0 ** -18 * Aa.max(axis=1)[:, None] * np.abs(X).max(axis=0)
    bz = (c + 2 * m * 2.0 ** -24) * (Aa.T @ np.abs(W)) + \
        2.0 ** -18 * (Aa.max(axis=1) @ np.abs(W)).max() * np.ones((1, l))
    assert np.all(np.abs(Y - Yo) <= by), float(np.max(np.abs(Y - Yo) / by))
    assert np.all(np.abs(Z - Zo) <= bz), float(np.max(np.abs(Z - Zo) / bz))
    # E4M3 rounding of both operands leaves ~5% relative error in Frobenius
    # norm (BF16 would leave ~0.15%), whatever K
    assert np.linalg.norm(Y - Yo) / np.linalg.norm(Yo) > 2.0 ** -7


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 1000, 20, 10, 2), (3000, 512, 100, 10, 2), (800, 300, 16, 8, 1),
                                       (400, 1200, 12, 6, 2)])
def test_fp8_sketch_rsvd_equal_error(rs, handle, m, n, k, p, q):
    """Mixed precision with FP8 sketch and power passes (FP32-accurate
    projection): ||A - U S V^T||_F <= 1.01 x the oracle's at the same (k, p, q)."""
    import torch
    if (m, n) == (2000, 1000):
        A = inputs.small_planted()
    else:
        A = inputs.planted(m, n, inputs.exp_spectrum(min(m, n), 2.0 / k), seed=m + n)
    d_o, U_o, V_o = oracle.rsvd(A, k, p=p, q=q, seed=3)
    err_o = np.sqrt(oracle.residual_fro2(A, U_o, d_o, V_o))
    d, U, V, info = rs.rsvdgb_rsvd(handle, to_dev(A), k, opts=rs.make_opts(p=p, q=q, seed=3, prec="fp8_sketch"))
    torch.cuda.synchronize()
    assert info.status == 0, info.as_dict()
    err = np.sqrt(oracle.residual_fro2(A, U.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64),
                                       V.cpu().numpy().astype(np.float64)))
    assert err <= 1.01 * err_o, (err, err_o)
    fa = oracle.fro2(A)
    assert abs(info.fro2_A - fa) <= 1e-5 * fa
