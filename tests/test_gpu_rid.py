"""Randomized interpolative and CUR decompositions (Algorithms id, rid and
rcur, Sec. 7) through the C ABI, against the FP64 oracle on the same data and
test matrix.

Pivot choices are integers decided by floating point, and the FP32 path may
break a near-tie differently from the FP64 oracle; so the GPU's pivots are
checked for validity by replaying them in the oracle (each chosen column's
trailing norm within 2 % of the step's largest), and the values that follow
from them (Z, U) are compared with the oracle's at the same pivots.  Column
and row gathers are bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs

pytestmark = pytest.mark.gpu

PIVOT_TOL = 2e-2


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


def planted(m, n, rate=1.0 / 20.0, seed=5):
    return inputs.planted(m, n, inputs.exp_spectrum(min(m, n), rate), seed=seed)


def check_pivots(X, piv):
    """Replay the pivots in the FP64 oracle: each choice within PIVOT_TOL of
    the best trailing norm of its step."""
    _, _, chosen, best = oracle.pqr(X, len(piv), force_piv=piv)
    assert np.all(chosen >= (1.0 - PIVOT_TOL) * best), np.min(chosen / best)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 300, 20, 10, 1), (1537, 261, 15, 5, 2), (800, 800, 30, 10, 0)])
def test_rid_matches_oracle(rs, handle, m, n, k, p, q):
    import torch
    A = planted(m, n)
    r = rs.rsvdgb_rid(handle, to_dev(A), k, opts=rs.make_opts(p=p, q=q, seed=3))
    torch.cuda.synchronize()
    assert r["info"].status == 0, r["info"].as_dict()
    J = r["J"].cpu().numpy()
    Z = r["Z"].cpu().numpy().astype(np.float64)
    C = r["C"].cpu().numpy()
    assert len(set(J.tolist())) == k
    np.testing.assert_array_equal(C, A[:, J])
    _, Bo = oracle.rqb(A, k, p=p, q=q, seed=3)
    check_pivots(Bo, J)
    J_o, Z_o = oracle.id_decomp(Bo, k, force_piv=J)
    assert rel(Z, Z_o) < 1e-3, rel(Z, Z_o)
    np.testing.assert_array_equal(Z[:, J], np.eye(k))
    # the same approximation quality as the oracle's own ID
    Co, Zo_own, _, _ = oracle.rid(A, k, p=p, q=q, seed=3)
    Av = A.astype(np.float64)
    e_gpu = np.linalg.norm(Av - C.astype(np.float64) @ Z)
    e_or = np.linalg.norm(Av - Co @ Zo_own)
    assert e_gpu <= 1.02 * e_or, (e_gpu, e_or)


def test_rid_exact_rank(rs, handle):
    import torch
    rng = np.random.default_rng(1)
    A = (rng.standard_normal((1200, 8)) @ rng.standard_normal((8, 200))).astype(np.float32)
    r = rs.rsvdgb_rid(handle, to_dev(A), 8, opts=rs.make_opts(p=4, q=1, seed=1))
    torch.cuda.synchronize()
    assert r["info"].status == 0
    C = r["C"].cpu().numpy().astype(np.float64)
    Z = r["Z"].cpu().numpy().astype(np.float64)
    assert rel(C @ Z, A.astype(np.float64)) < 1e-4


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 300, 20, 10, 1), (900, 500, 12, 8, 2)])
def test_rcur_matches_oracle(rs, handle, m, n, k, p, q):
    import torch
    A = planted(m, n, seed=9)
    r = rs.rsvdgb_rcur(handle, to_dev(A), k, opts=rs.make_opts(p=p, q=q, seed=4))
    torch.cuda.synchronize()
    assert r["info"].status == 0, r["info"].as_dict()
    J = r["J"].cpu().numpy()
    I = r["I"].cpu().numpy()
    C = r["C"].cpu().numpy()
    R = r["R"].cpu().numpy()
    U = r["U"].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(C, A[:, J])
    np.testing.assert_array_equal(R, A[I, :])
    assert len(set(I.tolist())) == k
    _, Bo = oracle.rqb(A, k, p=p, q=q, seed=4)
    check_pivots(Bo, J)
    check_pivots(np.ascontiguousarray(C.T.astype(np.float64)), I)
    _, Z_o = oracle.id_decomp(Bo, k, force_piv=J)
    U_o = Z_o @ np.linalg.pinv(R.astype(np.float64))
    assert rel(U, U_o) < 2e-3, rel(U, U_o)
    Av = A.astype(np.float64)
    e_gpu = np.linalg.norm(Av - C.astype(np.float64) @ U @ R.astype(np.float64))
    Co, Uo, Ro, _, _ = oracle.rcur(A, k, p=p, q=q, seed=4)
    e_or = np.linalg.norm(Av - Co @ Uo @ Ro)
    assert e_gpu <= 1.05 * e_or, (e_gpu, e_or)


def test_rid_layouts_dtypes_and_indices_only(rs, handle):
    import torch
    A = planted(1000, 240, seed=2)
    ref = rs.rsvdgb_rid(handle, to_dev(A), 10, opts=rs.make_opts(p=6, q=1, seed=2))
    # column-major storage of the same matrix: same indices and Z
    col = rs.rsvdgb_rid(handle, to_dev(A.T.copy()), 10, opts=rs.make_opts(p=6, q=1, seed=2, layout="col"))
    only = rs.rsvdgb_rid(handle, to_dev(A), 10, opts=rs.make_opts(p=6, q=1, seed=2), idx_only=True)
    torch.cuda.synchronize()
    _, Bo = oracle.rqb(A, 10, p=6, q=1, seed=2)
    Jc = col["J"].cpu().numpy()
    check_pivots(Bo, Jc)
    _, Z_o = oracle.id_decomp(Bo, 10, force_piv=Jc)
    assert rel(col["Z"].cpu().numpy().astype(np.float64), Z_o) < 1e-3
    np.testing.assert_array_equal(only["J"].cpu().numpy(), ref["J"].cpu().numpy())
    assert only["C"] is None and only["Z"] is None
    # BF16 storage: C holds the exact BF16 values of the chosen columns
    bits = inputs.bf16_bits(A)
    Ab = to_dev(bits.view(np.int16)).view(torch.bfloat16)
    rb = rs.rsvdgb_rid(handle, Ab, 10, opts=rs.make_opts(p=6, q=1, seed=2))
    torch.cuda.synchronize()
    assert rb["info"].status == 0
    Jb = rb["J"].cpu().numpy()
    np.testing.assert_array_equal(rb["C"].cpu().numpy(), inputs.bf16_to_f32(bits)[:, Jb])
    _, Bo = oracle.rqb(bits, 10, p=6, q=1, seed=2)
    check_pivots(Bo, Jb)


def test_rid_rcur_argument_errors(rs, handle):
    import ctypes
    import torch
    lib = rs.load()
    A = to_dev(planted(100, 300))  # m < n
    J = torch.empty(5, dtype=torch.int64, device="cuda")
    o = rs.make_opts()
    rc = lib.rsvdgb_rid(handle.ptr, A.data_ptr(), 100, 300, 300, 0, 5, ctypes.byref(o), None, 5, None, 300,
                        J.data_ptr(), None)
    assert rc == 7  # RSVDGB_ERR_UNSUPPORTED: the row ID is the column ID of A^T
    A2 = to_dev(planted(300, 100))
    rc = lib.rsvdgb_rid(handle.ptr, A2.data_ptr(), 300, 100, 100, 0, 5, ctypes.byref(o), None, 5, None, 100,
                        None, None)
    assert rc == rs.RSVDGB_ERR_INVALID_ARG
    rc = lib.rsvdgb_rcur(handle.ptr, A2.data_ptr(), 300, 100, 100, 0, 5, ctypes.byref(o), None, 5, None, 5, None,
                         100, J.data_ptr(), None, None)
    assert rc == rs.RSVDGB_ERR_INVALID_ARG


def test_rid_rcur_full_size_properties(rs, handle):
    """200000 x 2000 (the benchmark's matrix), k = 100, p = 10, q = 2: C and
    R are bit-exact gathers, Z(:, J) = I, the indices are distinct, and the
    ID / CUR errors stay within a small factor of the rank-k rSVD error of
    the same matrix (an ID is not optimal, Sec. 7)."""
    import torch
    m, n, k = 200000, 2000, 100
    A = inputs.spiked_noise(m, n, 1.0 / np.arange(1, n + 1), 1e-3, seed=0x160802148 + 2000, device="cuda")
    o = rs.make_opts(p=10, q=2, seed=2)
    r = rs.rsvdgb_rid(handle, A, k, opts=o)
    c = rs.rsvdgb_rcur(handle, A, k, opts=o)
    d, U, V, info = rs.rsvdgb_rsvd(handle, A, k, opts=o)
    torch.cuda.synchronize()
    assert r["info"].status == 0 and c["info"].status == 0 and info.status == 0
    J = r["J"]
    assert torch.unique(J).numel() == k and torch.unique(c["I"]).numel() == k
    assert torch.equal(r["C"], A[:, J])
    assert torch.equal(c["R"], A[c["I"], :])
    Z = r["Z"]
    assert torch.equal(Z[:, J], torch.eye(k, device="cuda"))
    A64 = A.double()
    e_svd = float(torch.linalg.matrix_norm(A64 - (U.double() * d.double()) @ V.double().T))
    e_id = float(torch.linalg.matrix_norm(A64 - r["C"].double() @ Z.double()))
    e_cur = float(torch.linalg.matrix_norm(A64 - c["C"].double() @ c["U"].double() @ c["R"].double()))
    assert e_svd <= e_id <= 3.0 * e_svd, (e_id, e_svd)
    assert e_svd <= e_cur <= 3.0 * e_svd, (e_cur, e_svd)


def test_rid_maximal_rank_and_rank_deficiency(rs, handle):
    """k = n - 1 with l = n (the sketch spans the whole row space): Z matches
    the oracle's at the same pivots.  A with only 5 nonzero columns and
    k = 8: a pivot step finds no direction left; the status says so, the
    missing indices are -1 and their columns of C are zero."""
    import torch
    A = planted(400, 40, seed=6)
    r = rs.rsvdgb_rid(handle, to_dev(A), 39, opts=rs.make_opts(p=5, q=1, seed=2))
    torch.cuda.synchronize()
    assert r["info"].status == 0
    J = r["J"].cpu().numpy()
    np.testing.assert_array_equal(r["C"].cpu().numpy(), A[:, J])
    _, Bo = oracle.rqb(A, 39, p=5, q=1, seed=2)
    check_pivots(Bo, J)
    _, Z_o = oracle.id_decomp(Bo, 39, force_piv=J)
    assert rel(r["Z"].cpu().numpy().astype(np.float64), Z_o) < 1e-3
    D = np.zeros((300, 60), np.float32)
    cols = [3, 17, 29, 41, 55]
    D[:, cols] = np.random.default_rng(0).standard_normal((300, 5))
    r2 = rs.rsvdgb_rid(handle, to_dev(D), 8, opts=rs.make_opts(p=4, q=1, seed=2))
    torch.cuda.synchronize()
    assert r2["info"].status == 4  # RSVDGB_ERR_BREAKDOWN
    J2 = r2["J"].cpu().numpy()
    C2 = r2["C"].cpu().numpy()
    assert np.all(J2[5:] == -1) and set(J2[J2 >= 0].tolist()) <= set(cols)
    np.testing.assert_array_equal(C2[:, J2 < 0], 0.0)
    np.testing.assert_array_equal(C2[:, J2 >= 0], D[:, J2[J2 >= 0]])


@pytest.mark.parametrize("m,n", [(3000, 400), (600, 64)])  # several CTAs; one CTA
def test_bounded_grid_barrier_wait_runs_out(rs, handle, m, n):
    """Failure detection without a device fault: the test hook leaves one
    CTA's arrival at the pivoted QR's first grid barrier out and bounds every
    wait by 2e6 clock ticks (about 1 ms).  The waits run out, the call reports
    RSVDGB_ERR_TIMEOUT in its info, the stream completes promptly, and the
    same handle then computes a correct rid (the context stays usable)."""
    import time
    import torch
    A = inputs.planted(m, n, inputs.exp_spectrum(n, 0.05), seed=m + n)
    A_dev = to_dev(A)
    opts = rs.make_opts(p=6, q=1, seed=4)
    rs.rsvdgb_test_pqr_barrier(handle, 2_000_000)
    t0 = time.perf_counter()
    r = rs.rsvdgb_rid(handle, A_dev, 10, opts=opts)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert r["info"].status == 6, r["info"].as_dict()  # RSVDGB_ERR_TIMEOUT
    # the hook was consumed: the next call runs normally on the same handle
    r2 = rs.rsvdgb_rid(handle, A_dev, 10, opts=opts)
    torch.cuda.synchronize()
    assert r2["info"].status == 0
    J = r2["J"].cpu().numpy()
    assert len(set(J.tolist())) == 10 and J.min() >= 0 and J.max() < n
    d_o, _, _ = oracle.rsvd(A, 10, p=6, q=1, seed=4)
    C, Z = r2["C"].cpu().numpy().astype(np.float64), r2["Z"].cpu().numpy().astype(np.float64)
    # an interpolative decomposition of rank 10 within a few times the optimum
    opt = np.sqrt(np.sum(inputs.exp_spectrum(n, 0.05)[10:] ** 2))
    assert np.linalg.norm(A - C @ Z) <= 20 * opt
    with pytest.raises(rs.RsvdgbError):
        rs.rsvdgb_test_pqr_barrier(handle, 0)
