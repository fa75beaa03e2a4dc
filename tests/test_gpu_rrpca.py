"""Randomized robust PCA (Algorithm rrpca, Sec. 5) through the C ABI against
the FP64 oracle: same readings, same test matrices per iteration.  The
iterates differ by FP32 rounding, so the comparison is on the converged L and
S (and on the recovery of the planted low-rank and sparse parts), within
10^-3 relative, with iteration counts within a few of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("m,n,rank,density", [(300, 300, 5, 0.2), (2000, 400, 8, 0.1), (250, 700, 6, 0.05)])
def test_rrpca_matches_oracle_and_recovers(rs, handle, m, n, rank, density):
    import torch
    L0, S0, A64 = inputs.low_rank_plus_sparse(m, n, rank, density, seed=11)
    A = A64.astype(np.float32)
    r = rs.rsvdgb_rrpca(handle, torch.from_numpy(A).cuda(), opts=rs.make_opts(p=10, q=2, seed=3))
    torch.cuda.synchronize()
    res = r["result"]
    assert res.status == 0
    assert res.err < 1e-5
    ref = oracle.rrpca(A, p=10, q=2, seed=3)
    assert abs(res.iters - ref["iters"]) <= 3, (res.iters, ref["iters"])
    assert res.rank == rank
    L = r["L"].cpu().numpy().astype(np.float64)
    S = r["S"].cpu().numpy().astype(np.float64)
    assert rel(L, ref["L"]) < 1e-3, rel(L, ref["L"])
    assert rel(S, ref["S"]) < 1e-3, rel(S, ref["S"])
    assert rel(L, L0) < 1e-3 and rel(S, S0) < 1e-3, (rel(L, L0), rel(S, S0))
    Av = A.astype(np.float64)
    assert np.linalg.norm(Av - L - S) <= 2e-5 * np.linalg.norm(Av)


def test_rrpca_without_L_and_argument_errors(rs, handle):
    import ctypes
    import torch
    _, _, A64 = inputs.low_rank_plus_sparse(200, 150, 4, 0.1, seed=2)
    A = torch.from_numpy(A64.astype(np.float32)).cuda()
    r = rs.rsvdgb_rrpca(handle, A, want_L=False, opts=rs.make_opts(seed=1))
    full = rs.rsvdgb_rrpca(handle, A, opts=rs.make_opts(seed=1))
    torch.cuda.synchronize()
    assert r["L"] is None
    assert torch.equal(r["S"], full["S"])
    lib = rs.load()
    ro = rs.make_rrpca_opts()
    o = rs.make_opts(layout="col")
    S = torch.empty(200, 150, device="cuda")
    res = rs.RsvdgbRrpcaResult()
    rc = lib.rsvdgb_rrpca(handle.ptr, A.data_ptr(), 200, 150, 150, ctypes.byref(ro), ctypes.byref(o), None, 150,
                          S.data_ptr(), 150, ctypes.byref(res))
    assert rc == 7  # RSVDGB_ERR_UNSUPPORTED: row-major input only
    o = rs.make_opts()
    rc = lib.rsvdgb_rrpca(handle.ptr, A.data_ptr(), 200, 150, 150, ctypes.byref(ro), ctypes.byref(o), None, 150,
                          None, 150, ctypes.byref(res))
    assert rc == rs.RSVDGB_ERR_INVALID_ARG


def test_rrpca_the_papers_simulation_case(rs, handle):
    """Sec. 5.5: 300 x 300, rank 5, 20 % of the entries uniform on [-500, 500]."""
    import torch
    L0, S0, A64 = inputs.rrpca_example(4)
    A = A64.astype(np.float32)
    r = rs.rsvdgb_rrpca(handle, torch.from_numpy(A).cuda(), opts=rs.make_opts(p=10, q=2, seed=3))
    torch.cuda.synchronize()
    res = r["result"]
    assert res.status == 0 and res.err < 1e-5 and res.rank == 5
    ref = oracle.rrpca(A, p=10, q=2, seed=3)
    L = r["L"].cpu().numpy().astype(np.float64)
    S = r["S"].cpu().numpy().astype(np.float64)
    tol_L = 10 * 1e-5 * np.linalg.norm(A64) / np.linalg.norm(L0)
    assert rel(L, ref["L"]) < tol_L and rel(L, L0) < tol_L, (rel(L, ref["L"]), rel(L, L0), tol_L)
    assert rel(S, ref["S"]) < 1e-4 and rel(S, S0) < 1e-4


def test_rrpca_iteration_cap_and_zero_matrix(rs, handle):
    import torch
    _, _, A64 = inputs.low_rank_plus_sparse(200, 150, 4, 0.1, seed=2)
    A = torch.from_numpy(A64.astype(np.float32)).cuda()
    r = rs.rsvdgb_rrpca(handle, A, ropts=rs.make_rrpca_opts(maxiter=1), opts=rs.make_opts(seed=1))
    torch.cuda.synchronize()
    assert r["result"].iters == 1 and r["result"].status == 0 and r["result"].err > 1e-5
    with pytest.raises(rs.RsvdgbError) as e:
        rs.rsvdgb_rrpca(handle, torch.zeros(100, 80, device="cuda"))
    assert e.value.status == rs.RSVDGB_ERR_INVALID_ARG
    An = A.clone()
    An[17, 4] = float("nan")
    with pytest.raises(rs.RsvdgbError) as e:
        rs.rsvdgb_rrpca(handle, An)
    assert e.value.status == 5  # RSVDGB_ERR_NONFINITE
