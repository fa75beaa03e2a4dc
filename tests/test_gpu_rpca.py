"""Randomized PCA (Algorithm rpca, Sec. 4.2, with the centring / scaling of
the rpca() interface, Sec. 4.4) through the C ABI, against the FP64 oracle on
the same data and the same test matrix.

Tolerances follow the FP32 rSVD bar applied to X = (A - 1 mu^T) diag(1/s):
the standard deviations sdev = sigma / sqrt(m - 1) within 1e-5 sdev_1 of the
oracle's (the singular-value bar), the rotation's and scores' spans within the
gap-ruled subspace tolerance, centre and scale to FP32 rounding of the FP64
statistics.  The implicit centring costs one FP32 rounding of mu against the
products with A, so the data keep the column offsets a few spreads from zero
(mean_ratio 5), as real measurements with units do.
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


def check_rpca(rs, handle, A_np, k, p=10, q=2, center=True, scale=True, layout="row", dtype="f32", seed=0,
               engine="auto", retx=True, sd_tol=1e-5):
    import torch
    if dtype == "bf16":
        A_or = inputs.bf16_bits(A_np)
        A_dev = to_dev(A_or.view(np.int16)).view(torch.bfloat16)
    else:
        A_or = A_np
        A_dev = to_dev(A_np)
    m, n = A_np.shape
    ref = oracle.rpca(A_or, k, center=center, scale=scale, p=p, q=q, seed=seed)
    opts = rs.make_opts(p=p, q=q, seed=seed, layout=layout, engine=engine)
    if layout == "col":
        A_dev = A_dev.t().contiguous()
    r = rs.rsvdgb_rpca(handle, A_dev, k, center=center, scale=scale, retx=retx, opts=opts)
    torch.cuda.synchronize()
    info = r["info"]
    assert info.status == 0, info.as_dict()
    sd = r["sdev"].cpu().numpy().astype(np.float64)
    eig = r["eigvals"].cpu().numpy().astype(np.float64)
    assert sigma_err(sd, ref["sdev"]) <= sd_tol, (sigma_err(sd, ref["sdev"]), sd[:4], ref["sdev"][:4])
    np.testing.assert_allclose(eig, sd ** 2, rtol=1e-5)
    assert np.all(np.diff(eig) <= 1e-6 * eig[0])
    # gap rule from the oracle's spectrum of B for the analysed matrix X
    _, _, _, _, Bo = oracle.rsvd(ref["X"], k, p=p, q=q, seed=seed, return_qb=True)
    sB = np.linalg.svd(Bo, compute_uv=False)
    tol = subspace_tol(sB, k, sB[0])
    W = r["rotation"].cpu().numpy()
    assert sin_theta(W, ref["rotation"]) <= tol, (sin_theta(W, ref["rotation"]), tol)
    assert np.max(np.abs(W.T @ W - np.eye(k))) < 1e-4
    if retx:
        Z = r["x"].cpu().numpy().astype(np.float64)
        assert sin_theta(Z, ref["x"]) <= tol, (sin_theta(Z, ref["x"]), tol)
        # Z = U Sigma: orthogonal columns of norm sigma = sdev sqrt(m - 1)
        ZtZ = Z.T @ Z
        sig = ref["sigma"]
        assert np.max(np.abs(np.sqrt(np.diag(ZtZ)) - sig)) <= 1e-5 * sig[0]
        off = ZtZ - np.diag(np.diag(ZtZ))
        assert np.max(np.abs(off)) <= 1e-4 * sig[0] ** 2
    else:
        assert r["x"] is None
    mu = r["center"].cpu().numpy()
    sc = r["scale"].cpu().numpy()
    spread = np.maximum(np.abs(ref["center"]), ref["scale"])
    assert np.all(np.abs(mu - ref["center"]) <= 2e-6 * spread), np.max(np.abs(mu - ref["center"]) / spread)
    np.testing.assert_allclose(sc, ref["scale"], rtol=2e-6, atol=1e-30)
    fx = float(np.sum(ref["X"] ** 2))
    assert abs(info.fro2_A - fx) <= 1e-5 * fx
    return r, ref


def data(m, n, rank=12, seed=21, **kw):
    return inputs.pca_data(m, n, rank, seed=seed, **kw).numpy()


@pytest.mark.parametrize("m,n,k,p,q", [
    (2000, 300, 10, 10, 2), (1537, 261, 20, 5, 1), (700, 130, 5, 5, 0),
])
def test_rpca_correlation(rs, handle, m, n, k, p, q):
    check_rpca(rs, handle, data(m, n), k, p=p, q=q)


@pytest.mark.parametrize("center,scale", [(True, False), (False, True), (False, False)])
def test_rpca_preprocessing_variants(rs, handle, center, scale):
    check_rpca(rs, handle, data(1200, 200), 8, p=8, q=1, center=center, scale=scale)


@pytest.mark.parametrize("layout", ["row", "col"])
def test_rpca_more_variables_than_observations(rs, handle, layout):
    """m < n: the variables are the rows of the logical (transposed) problem."""
    check_rpca(rs, handle, data(300, 900), 12, p=8, q=2, layout=layout)


def test_rpca_column_major(rs, handle):
    check_rpca(rs, handle, data(900, 250), 10, p=10, q=1, layout="col")


def test_rpca_bf16_data(rs, handle):
    check_rpca(rs, handle, data(1500, 320), 10, p=10, q=2, dtype="bf16")


def test_rpca_simt_engine(rs, handle):
    check_rpca(rs, handle, data(800, 150), 6, p=6, q=1, engine="simt")


def test_rpca_constant_column_and_no_scores(rs, handle):
    r, ref = check_rpca(rs, handle, data(1000, 180, zero_var_cols=2), 8, p=8, q=1, retx=False)
    sc = r["scale"].cpu().numpy()
    assert np.all(sc[-2:] == 0.0)
    W = r["rotation"].cpu().numpy()
    assert np.max(np.abs(W[-2:])) == 0.0


def test_rpca_host_entry_point_matches_device(rs, handle):
    import torch
    A = data(1100, 210)
    opts = rs.make_opts(p=10, q=2, seed=5)
    r_d = rs.rsvdgb_rpca(handle, to_dev(A), 9, opts=opts)
    torch.cuda.synchronize()
    r_h = rs.rsvdgb_rpca_host(handle, torch.from_numpy(A).pin_memory(), 9, opts=opts)
    assert r_h["info"].status == 0
    for key in ("eigvals", "sdev", "rotation", "x", "center", "scale"):
        np.testing.assert_array_equal(r_h[key].numpy(), r_d[key].cpu().numpy())


def test_rpca_invalid_arguments(rs, handle):
    import ctypes
    import torch
    lib = rs.load()
    A = to_dev(data(100, 20))
    eig = torch.empty(5, device="cuda")
    rot = torch.empty(20, 5, device="cuda")
    o = rs.make_opts()
    # eigvals NULL
    rc = lib.rsvdgb_rpca(handle.ptr, A.data_ptr(), 100, 20, 20, 0, 5, 1, 1, ctypes.byref(o), rot.data_ptr(), 5,
                         None, None, None, 5, None, None, None)
    assert rc == rs.RSVDGB_ERR_INVALID_ARG
    # rotation leading dimension < k
    rc = lib.rsvdgb_rpca(handle.ptr, A.data_ptr(), 100, 20, 20, 0, 5, 1, 1, ctypes.byref(o), rot.data_ptr(), 4,
                         eig.data_ptr(), None, None, 5, None, None, None)
    assert rc == rs.RSVDGB_ERR_INVALID_ARG
    # k >= min(m, n)
    rc = lib.rsvdgb_rpca(handle.ptr, A.data_ptr(), 100, 20, 20, 0, 20, 1, 1, ctypes.byref(o), None, 20,
                         eig.data_ptr(), None, None, 20, None, None, None)
    assert rc == rs.RSVDGB_ERR_INVALID_ARG


def test_rpca_full_size_properties(rs, handle):
    """200000 x 2000 data, k = 100, p = 10, q = 2 (the size the benchmark
    times): centre and scale against FP64 column statistics of the stored
    values; scores with zero column means and orthogonal columns of norm
    sigma; orthonormal rotation; ||X||_F^2 = (m - 1) n for correlation PCA."""
    import torch
    m, n, k = 200000, 2000, 100
    A = inputs.pca_data(m, n, 100, seed=0x160802148 + 6000, device="cuda")
    r = rs.rsvdgb_rpca(handle, A, k, opts=rs.make_opts(p=10, q=2, seed=1))
    torch.cuda.synchronize()
    info = r["info"]
    assert info.status == 0
    Ad = A.double()
    mu = Ad.mean(dim=0)
    sd = Ad.std(dim=0, correction=1)
    del Ad
    mu_g = r["center"].double()
    sc_g = r["scale"].double()
    assert float(torch.max(torch.abs(mu_g - mu) / torch.maximum(mu.abs(), sd))) <= 2e-6
    assert float(torch.max(torch.abs(sc_g - sd) / sd)) <= 2e-6
    assert abs(info.fro2_A - (m - 1) * n) <= 1e-5 * (m - 1) * n
    Z = r["x"].double()
    eig = r["eigvals"].double()
    sig = torch.sqrt(eig * (m - 1))
    colsum = Z.sum(dim=0)
    assert float(torch.max(torch.abs(colsum))) <= 1e-4 * float(sig[0]) * m ** 0.5
    ZtZ = Z.T @ Z
    assert float(torch.max(torch.abs(torch.sqrt(torch.diag(ZtZ)) - sig))) <= 1e-5 * float(sig[0])
    off = ZtZ - torch.diag(torch.diag(ZtZ))
    assert float(torch.max(torch.abs(off))) <= 1e-4 * float(sig[0]) ** 2
    W = r["rotation"].double()
    assert float(torch.max(torch.abs(W.T @ W - torch.eye(k, dtype=torch.float64, device="cuda")))) <= 1e-4
    assert float(eig.sum()) <= n * (1 + 1e-5)
    assert bool(torch.all(eig[1:] <= eig[:-1] * (1 + 1e-6)))


def test_rpca_maximal_rank(rs, handle):
    """k = n - 1: the sketch spans all variables, so rpca returns the exact
    leading principal components (numpy's correlation eigenvalues)."""
    import torch
    A = data(500, 30)
    r = rs.rsvdgb_rpca(handle, to_dev(A), 29, opts=rs.make_opts(p=5, q=1, seed=4))
    torch.cuda.synchronize()
    assert r["info"].status == 0
    w = np.linalg.eigvalsh(np.corrcoef(A.astype(np.float64).T))[::-1]
    eig = r["eigvals"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(eig - w[:29])) <= 5e-5 * w[0], np.max(np.abs(eig - w[:29])) / w[0]
    W = r["rotation"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(W.T @ W - np.eye(29))) < 1e-4
