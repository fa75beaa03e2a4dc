"""Batched rSVD (one graph launch over many ragged matrices) against the FP64
oracle, matrix by matrix, through the C ABI."""
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


def test_batched_matches_oracle_per_matrix(rs):
    import torch
    rng_shapes = inputs.ragged_shapes(24, (70, 700), (40, 400), seed=5)
    ms, ns, rates = rng_shapes
    # include wide matrices (m < n) and exact multiples of the block sizes
    ms[0], ns[0] = 128, 64
    ms[1], ns[1] = 60, 300
    ms[2], ns[2] = 257, 129
    mats, _ = inputs.ragged_batch(24, seed=9, device="cuda", shapes=(ms, ns, rates))
    k, p, q = 8, 6, 1
    h = rs.Handle(0)
    try:
        call = rs.BatchedCall(mats, k)
        rs.rsvdgb_rsvd_batched(h, call, rs.make_opts(p=p, q=q, seed=11))
        torch.cuda.synchronize()
        # a second call with the same layout replays the cached graph
        rs.rsvdgb_rsvd_batched(h, call, rs.make_opts(p=p, q=q, seed=11))
        torch.cuda.synchronize()
        for b, A in enumerate(mats):
            An = A.cpu().numpy()
            d_o, U_o, V_o, Q_o, B_o = oracle.rsvd(An, k, p=p, q=q, seed=11, return_qb=True)
            info = call.info(b)
            assert info.status == 0, (b, info.as_dict())
            d = call.d[b].cpu().numpy()
            assert sigma_err(d, d_o) <= 1e-5, (b, An.shape, sigma_err(d, d_o))
            sB = np.linalg.svd(B_o, compute_uv=False)
            tol = subspace_tol(sB, k, sB[0])
            assert sin_theta(call.U[b].cpu().numpy(), U_o) <= tol, (b, An.shape)
            assert sin_theta(call.V[b].cpu().numpy(), V_o) <= tol, (b, An.shape)
            fa = oracle.fro2(An)
            assert abs(info.fro2_A - fa) <= 1e-5 * fa
    finally:
        h.close()


def test_batched_rejects_wide_sketch(rs):
    import torch
    mats = [torch.randn(100, 80, device="cuda")]
    h = rs.Handle(0)
    try:
        call = rs.BatchedCall(mats, 30)
        with pytest.raises(rs.RsvdgbError) as e:
            rs.rsvdgb_rsvd_batched(h, call, rs.make_opts(p=10, q=1))
        assert e.value.status == 7  # l = 40 > 32
    finally:
        h.close()


def test_batched_full_size_workload_sampled(rs):
    """The batched workload the benchmark times: 4096 matrices, m log-uniform
    in [256, 4096], n in [64, 1024], exponential spectra with decay rates in
    [0.05, 0.5], k = 16, p = 8, q = 1, one graph launch.  Every matrix reports
    status 0 and ||A||_F^2 within 1e-5; against the oracle, one by one: the
    tallest matrices with the fastest decay (where FP32 rounding along the
    rows meets a large sigma_1 / sigma_l) and a seeded random sample, all
    under the same sigma and gap-rule tolerances as the single-matrix path."""
    import torch
    count, k, p, q = 4096, 16, 8, 1
    mats, rates = inputs.ragged_batch(count, seed=0x160802148 + 4000, device="cuda")
    h = rs.Handle(0)
    try:
        call = rs.BatchedCall(mats, k)
        rs.rsvdgb_rsvd_batched(h, call, rs.make_opts(p=p, q=q, seed=3))
        torch.cuda.synchronize()
        fro = torch.stack([(A.double() ** 2).sum() for A in mats]).cpu().numpy()
        for b in range(count):
            info = call.info(b)
            assert info.status == 0, (b, info.as_dict())
            assert abs(info.fro2_A - fro[b]) <= 1e-5 * fro[b], b
        shapes = np.array([A.shape for A in mats])
        rates = np.asarray(rates)
        hard = np.argsort(-(shapes[:, 0] * rates))[:16]  # tall and fast-decaying
        rng = np.random.default_rng(4000)
        sample = np.unique(np.concatenate([hard, rng.choice(count, 24, replace=False)]))
        for b in sample.tolist():
            An = mats[b].cpu().numpy()
            d_o, U_o, V_o, Q_o, B_o = oracle.rsvd(An, k, p=p, q=q, seed=3, return_qb=True)
            d = call.d[b].cpu().numpy()
            assert sigma_err(d, d_o) <= 1e-5, (b, An.shape, rates[b], sigma_err(d, d_o))
            sB = np.linalg.svd(B_o, compute_uv=False)
            tol = subspace_tol(sB, k, sB[0])
            su = sin_theta(call.U[b].cpu().numpy(), U_o)
            sv = sin_theta(call.V[b].cpu().numpy(), V_o)
            assert su <= tol and sv <= tol, (b, An.shape, rates[b], su, sv, tol)
    finally:
        h.close()
