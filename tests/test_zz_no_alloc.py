"""The allocation-free A^T X entry point (for callers that cannot allocate
device memory while they run) against the regular entry point, through the C
ABI, on two calls in a row.  Collected last so that a failure here stops a
-x run only after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_atx_matches_regular_entry_point_twice():
    import torch
    from paper_1608_02148_gb300 import build, rsvdgb as rs

    build.build()
    h = rs.Handle(0)
    try:
        rng = np.random.default_rng(20261203)
        for m, n, l in ((5000, 700, 40), (3001, 257, 110)):  # two calls in a row, different shapes
            A = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
            X = torch.from_numpy(rng.standard_normal((m, l)).astype(np.float32)).cuda()
            Z_ref = rs.rsvdgb_pass_atx(h, A, X, engine="simt")
            Z = torch.full((n, l), float("nan"), dtype=torch.float32, device="cuda")
            rs.rsvdgb_pass_atx_noalloc(A, X, Z)
            torch.cuda.synchronize()
            Zr = Z_ref.cpu().numpy().astype(np.float64)
            Zn = Z.cpu().numpy().astype(np.float64)
            # the FP32 accumulation bound used by the pass parity tests
            bound = 2 * m * 2.0 ** -24 * (np.abs(A.cpu().numpy()).T.astype(np.float64) @ np.abs(X.cpu().numpy()))
            assert np.all(np.isfinite(Zn))
            assert np.all(np.abs(Zn - Zr) <= 2 * bound)
        # a problem larger than the static scratch is rejected before any work
        big_n = rs.NOALLOC_SCRATCH_BYTES // (4 * 64) + 1
        A = torch.zeros(4, big_n, device="cuda")
        X = torch.zeros(4, 64, device="cuda")
        with pytest.raises(ValueError):
            rs.rsvdgb_pass_atx_noalloc(A, X)
        rc = rs.load().rsvdgb_pass_atx_noalloc(None, A.data_ptr(), 4, big_n, big_n, 0, X.data_ptr(), 64, 64,
                                               X.data_ptr(), 64)
        assert rc == 1
    finally:
        h.close()


def test_noalloc_atx_rejects_bad_operands_before_queueing():
    """Wrong shapes, dtypes, strides or devices of X and Z raise in the binding
    before the C call, so nothing is queued and nothing is written."""
    import torch
    from paper_1608_02148_gb300 import build, rsvdgb as rs

    build.build()
    m, n, l = 300, 40, 8
    A = torch.randn(m, n, device="cuda")
    X = torch.randn(m, l, device="cuda")
    bad_z = [
        torch.zeros(n - 1, l, device="cuda"),                       # too few rows
        torch.zeros(n, l + 1, device="cuda"),                       # too many columns
        torch.zeros(n, l, dtype=torch.bfloat16, device="cuda"),     # not float32
        torch.zeros(l, n, device="cuda").t(),                       # column stride not 1
        torch.zeros(n, l),                                          # on the host
    ]
    for Z in bad_z:
        before = Z.clone()
        with pytest.raises(ValueError):
            rs.rsvdgb_pass_atx_noalloc(A, X, Z)
        assert torch.equal(Z, before)
    for Xb in (torch.randn(m + 1, l, device="cuda"), X.to(torch.bfloat16), X.cpu()):
        with pytest.raises(ValueError):
            rs.rsvdgb_pass_atx_noalloc(A, Xb)
    with pytest.raises(ValueError):
        rs.rsvdgb_pass_atx_noalloc(A.cpu(), X.cpu())
    torch.cuda.synchronize()
