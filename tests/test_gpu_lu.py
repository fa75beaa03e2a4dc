"""Normalized power iterations (Algorithm norm_iterations, Sec. 2.2.2) on the
GPU against the oracle's, through the C ABI.

The GPU picks its pivot rows by tournament pivoting and the oracle by partial
pivoting over all rows, so the L factors differ; both span the sketch, so the
rSVDs agree within the FP32 tolerances (sigma within 1e-5 sigma_1, U_k and
V_k within the gap rule of the oracle's spectrum of B)."""
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


def _check(rs, handle, A, k, p, q, seed):
    import torch
    d_o, U_o, V_o, Q_o, B_o = oracle.rsvd(A, k, p=p, q=q, seed=seed, return_qb=True, scheme="lu")
    d, U, V, info = rs.rsvdgb_rsvd(handle, to_dev(A), k, opts=rs.make_opts(p=p, q=q, seed=seed, power="lu"))
    torch.cuda.synchronize()
    assert info.status == 0, info.as_dict()
    d, U, V = d.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
    assert sigma_err(d, d_o) <= 1e-5, sigma_err(d, d_o)
    sB = np.linalg.svd(B_o, compute_uv=False)
    tol = subspace_tol(sB, k, sB[0])
    assert sin_theta(U, U_o) <= tol and sin_theta(V, V_o) <= tol, (sin_theta(U, U_o), sin_theta(V, V_o), tol)
    return d, U, V


def test_lu_scheme_small_planted(rs, handle):
    """2000 x 1000, sigma_i = exp(-i/20), k = 20, p = 10, q = 2."""
    _check(rs, handle, inputs.small_planted(), 20, 10, 2, 0)


@pytest.mark.parametrize("m,n,k,p,q", [(5000, 700, 40, 10, 3), (1030, 512, 100, 12, 1), (4000, 64, 10, 6, 2),
                                       (300, 260, 50, 10, 2)])
def test_lu_scheme_ragged(rs, handle, m, n, k, p, q):
    sigma = inputs.exp_spectrum(min(m, n), 3.0 / min(m, n))
    _check(rs, handle, inputs.planted(m, n, sigma, seed=m + 5 * n), k, p, q, m)


def test_lu_scheme_wide_and_column_major(rs, handle):
    """m < n runs on the transpose, like the subspace scheme."""
    import torch
    A = inputs.planted(400, 1500, inputs.exp_spectrum(400, 0.03), seed=21)
    d_o, U_o, V_o = oracle.rsvd(A, 15, p=8, q=2, seed=6, scheme="lu")
    d, U, V, info = rs.rsvdgb_rsvd(handle, to_dev(A), 15, opts=rs.make_opts(p=8, q=2, seed=6, power="lu"))
    torch.cuda.synchronize()
    assert info.status == 0
    assert sigma_err(d.cpu().numpy(), d_o) <= 1e-5


def test_lu_scheme_without_iterations_is_the_plain_sketch(rs, handle):
    import torch
    A = to_dev(inputs.planted(3000, 500, inputs.exp_spectrum(500, 0.02), seed=8))
    r1 = rs.rsvdgb_rsvd(handle, A, 25, opts=rs.make_opts(p=10, q=0, seed=1, power="lu"))
    r0 = rs.rsvdgb_rsvd(handle, A, 25, opts=rs.make_opts(p=10, q=0, seed=1))
    torch.cuda.synchronize()
    for a, b in zip(r0[:3], r1[:3]):
        assert torch.equal(a, b)


def test_lu_scheme_rejects_wide_sketches(rs, handle):
    import torch
    A = torch.randn(2000, 500, device="cuda")
    with pytest.raises(rs.RsvdgbError) as e:
        rs.rsvdgb_rsvd(handle, A, 120, opts=rs.make_opts(p=10, q=1, power="lu"))
    assert e.value.status == 7
