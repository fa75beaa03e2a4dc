"""End-to-end parity at the sizes the benchmark times, against the FP64 oracle
run on the same stored matrix and the same Philox test matrix.

* 200000 x 2000 FP32, sigma_i = 1/i planted under N(0, 1e-3^2) noise, k = 100,
  p = 10, q = 2: the FP32 path (the launch configuration of the benchmark:
  default engine and precision) element by element against the oracle --
  sigma within 1e-5 sigma_1, U_k and V_k within the gap rule of the oracle's
  spectrum of B, and Q over the whole l-space within max(1e-4, 10 u32 kappa(B));
  the BF16-sketch and FP8-sketch forms at equal reconstruction error (<= 1.01x
  the oracle's ||A - U S V^T||_F).
* A scaled case of the BF16-stored step-spectrum workload (20000 x 5000,
  sigma = 1 for i <= 200 and 1e-2 beyond, N(0, 1e-4^2) noise, k = 200, p = 20,
  q = 3): the FP32-accurate path against the same tolerances, the mixed form
  at equal error.
The oracle runs once per matrix (about ten seconds on the host cores each).
"""
import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs
from tests.helpers import U32, sigma_err, sin_theta, subspace_tol

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


def _oracle_case(A_host, k, p, q, seed):
    """The oracle's d, U, V, Q, B and its reconstruction error on A_host."""
    d, U, V, Q, B = oracle.rsvd(A_host, k, p=p, q=q, seed=seed, return_qb=True)
    err = np.sqrt(max(oracle.residual_fro2(A_host, U, d, V), 0.0))
    return dict(d=d, U=U, V=V, Q=Q, B=B, sB=np.linalg.svd(B, compute_uv=False), err=err)


def _check_fp32(rs, handle, A_dev, A_host, ref, k, p, q, seed, prec="fp32"):
    import torch
    opts = rs.make_opts(p=p, q=q, seed=seed, prec=prec)
    d, U, V, info = rs.rsvdgb_rsvd(handle, A_dev, k, opts=opts)
    Q, _, info_q = rs.rsvdgb_rqb(handle, A_dev, k, opts=opts)
    torch.cuda.synchronize()
    assert info.status == 0 and info_q.status == 0, info.as_dict()
    d, U, V, Q = (t.cpu().numpy() for t in (d, U, V, Q))
    sB = ref["sB"]
    assert sigma_err(d, ref["d"]) <= 1e-5, sigma_err(d, ref["d"])
    tol = subspace_tol(sB, k, sB[0])
    su, sv = sin_theta(U, ref["U"]), sin_theta(V, ref["V"])
    assert su <= tol and sv <= tol, (su, sv, tol)
    tol_q = max(1e-4, 10 * U32 * sB[0] / sB[-1])
    sq = sin_theta(Q, ref["Q"])
    assert sq <= tol_q, (sq, tol_q)
    assert np.max(np.abs(U.T.astype(np.float64) @ U - np.eye(k))) < 1e-4
    assert np.max(np.abs(V.T.astype(np.float64) @ V - np.eye(k))) < 1e-4
    return d, U, V, info


def _check_equal_error(rs, handle, A_dev, A_host, ref, k, p, q, seed, prec):
    import torch
    opts = rs.make_opts(p=p, q=q, seed=seed, prec=prec)
    d, U, V, info = rs.rsvdgb_rsvd(handle, A_dev, k, opts=opts)
    torch.cuda.synchronize()
    assert info.status == 0, info.as_dict()
    d, U, V = (t.cpu().numpy().astype(np.float64) for t in (d, U, V))
    err = np.sqrt(max(oracle.residual_fro2(A_host, U, d, V), 0.0))
    assert err <= 1.01 * ref["err"], (err, ref["err"])
    return err


@pytest.fixture(scope="module")
def spiked200k(rs):
    import torch
    m, n, k, p, q = 200000, 2000, 100, 10, 2
    sigma = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    A = inputs.spiked_noise(m, n, sigma, 1e-3, 0x160802148 + 2000, device="cuda")
    torch.cuda.synchronize()
    A_host = A.cpu().numpy()
    return A, A_host, _oracle_case(A_host, k, p, q, seed=0), (k, p, q)


def test_spiked_200000x2000_fp32_matches_oracle(rs, handle, spiked200k):
    A, A_host, ref, (k, p, q) = spiked200k
    _check_fp32(rs, handle, A, A_host, ref, k, p, q, seed=0)


@pytest.mark.parametrize("prec", ["bf16_sketch", "fp8_sketch"])
def test_spiked_200000x2000_mixed_at_equal_error(rs, handle, spiked200k, prec):
    A, A_host, ref, (k, p, q) = spiked200k
    _check_equal_error(rs, handle, A, A_host, ref, k, p, q, seed=0, prec=prec)


@pytest.fixture(scope="module")
def step20k(rs):
    import torch
    m, n, k, p, q = 20000, 5000, 200, 20, 3
    A = inputs.step_noise(m, n, 200, 1e-4, 0x160802148 + 3000, device="cuda", bf16=True)
    torch.cuda.synchronize()
    bits = A.view(torch.int16).cpu().numpy().view(np.uint16)
    return A, bits, _oracle_case(bits, k, p, q, seed=1), (k, p, q)


def test_step_bf16_20000x5000_fp32_matches_oracle(rs, handle, step20k):
    A, bits, ref, (k, p, q) = step20k
    _check_fp32(rs, handle, A, bits, ref, k, p, q, seed=1)


@pytest.mark.parametrize("prec", ["bf16_sketch", "fp8_sketch"])
def test_step_bf16_20000x5000_mixed_at_equal_error(rs, handle, step20k, prec):
    A, bits, ref, (k, p, q) = step20k
    _check_equal_error(rs, handle, A, bits, ref, k, p, q, seed=1, prec=prec)
