"""The learned (q, p) controller on the GPU, through the C ABI: the network's
forward pass and gradient against the FP64 oracle, the features against the
oracle's statement of them, the learned mode of rSVD against the oracle at the
(q, p) it chose, training, and what a trained controller gains over the
fixed p = 10, q = 2 of Sec. 3.4."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1608_02148_gb300 import inputs
from tests.helpers import sigma_err, sin_theta, subspace_tol

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEFAULT_CONTROLLER = os.path.join(ROOT, "paper_1608_02148_gb300", "controller_default.bin")


@pytest.fixture(scope="module")
def rs():
    import torch
    from paper_1608_02148_gb300 import build, rsvdgb
    build.build()
    assert torch.cuda.is_available()
    return rsvdgb


@pytest.fixture()
def handle(rs):
    h = rs.Handle(0)
    yield h
    h.close()


def random_params(rng, scale=0.3):
    P = rng.standard_normal(5410) * scale
    P[:16] = rng.standard_normal(16) * 0.1
    P[16:32] = np.abs(rng.standard_normal(16)) + 0.5
    return P


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_matches_oracle(rs, handle):
    rng = np.random.default_rng(0)
    P = random_params(rng).astype(np.float32)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    out = rs.rsvdgb_mlp_forward(handle, dev(P), dev(X)).cpu().numpy()
    ref = oracle.mlp_forward(P.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(out - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n,tau", [(333, 0.9), (64, 0.5), (1, 0.25)])
def test_gradient_matches_oracle(rs, handle, n, tau):
    """FP32 kernels against the FP64 reverse-mode gradient (itself pinned by
    finite differences): element-wise within 1e-4 of the gradient's scale."""
    rng = np.random.default_rng(n)
    P = random_params(rng).astype(np.float32)
    X = rng.standard_normal((n, 16)).astype(np.float32)
    Y = (rng.standard_normal((n, 2)) * 2).astype(np.float32)
    g, loss = rs.rsvdgb_mlp_grad(handle, dev(P), dev(X), dev(Y), tau)
    g = g.cpu().numpy()
    loss_o, g_o = oracle.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), tau)
    assert abs(float(loss.cpu()[0]) - loss_o) <= 1e-5 * max(1.0, abs(loss_o))
    scale = np.max(np.abs(g_o))
    assert np.max(np.abs(g - g_o)) <= 1e-4 * scale, np.max(np.abs(g - g_o)) / scale


def test_features_match_oracle(rs, handle):
    import torch
    A = inputs.planted(2000, 400, inputs.exp_spectrum(400, 1.0 / 40.0), seed=21)
    k, p_max = 20, 20
    opts = rs.make_opts(seed=4, p_max=p_max)
    f = rs.rsvdgb_controller_features(handle, dev(A), k, opts=opts)
    torch.cuda.synchronize()
    f = f.cpu().numpy().astype(np.float64)
    fo = oracle.controller_features(A, k, p_max=p_max, seed=4)
    assert np.max(np.abs(f - fo)) <= 1e-3, np.abs(f - fo)


def constant_controller(q, p):
    """A network whose output is its bias (q, log2 p), identity standardisation."""
    P = np.zeros(5410, np.float32)
    P[16:32] = 1.0
    P[-2:] = (q, math.log2(p))
    return P


def test_learned_mode_runs_the_chosen_q_and_p(rs, handle):
    """With a controller that always answers (q, p) = (1, 8), the learned mode
    must equal the oracle's rSVD at p = 8, q = 1: the first k + 8 columns of the
    widest sketch are the sketch for p = 8 (Omega nested in l)."""
    import torch
    rs.rsvdgb_controller_set(handle, constant_controller(1, 8))
    A = inputs.small_planted()
    k = 20
    d, U, V, info = rs.rsvdgb_rsvd(handle, dev(A), k, opts=rs.make_opts(q_mode="learned", p_max=40, seed=6))
    torch.cuda.synchronize()
    assert info.status == 0 and info.q_used == 1 and info.p_used == 8 and info.l == 28, info.as_dict()
    d_o, U_o, V_o, Q_o, B_o = oracle.rsvd(A, k, p=8, q=1, seed=6, return_qb=True)
    assert sigma_err(d.cpu().numpy(), d_o) <= 1e-5
    sB = np.linalg.svd(B_o, compute_uv=False)
    tol = subspace_tol(sB, k, sB[0])
    assert sin_theta(U.cpu().numpy(), U_o) <= tol
    assert sin_theta(V.cpu().numpy(), V_o) <= tol


def test_learned_mode_clamps_and_falls_back(rs, handle):
    import torch
    A = dev(inputs.planted(600, 200, inputs.exp_spectrum(200, 0.05), seed=2))
    # no controller loaded: the fixed (p, q) of the options
    d, U, V, info = rs.rsvdgb_rsvd(handle, A, 10, opts=rs.make_opts(p=5, q=3, q_mode="learned"))
    torch.cuda.synchronize()
    assert info.status == 0 and info.q_used == 3 and info.p_used == 5
    # a controller asking for more than allowed is clamped to q_max and p_max
    rs.rsvdgb_controller_set(handle, constant_controller(9, 64))
    d, U, V, info = rs.rsvdgb_rsvd(handle, A, 10, opts=rs.make_opts(q_mode="learned", p_max=30, q_max=4))
    torch.cuda.synchronize()
    assert info.status == 0 and info.q_used == 4 and info.p_used == 30


def test_training_fits_a_known_rule(rs, handle, tmp_path):
    """Targets that are a simple function of the features: the GPU-trained
    network's mean pinball loss ends far below that of its initial output, and
    its saved parameters give the same outputs in the oracle."""
    import struct
    import torch
    rng = np.random.default_rng(11)
    n = 2048
    X = rng.standard_normal((n, 16)).astype(np.float32)
    Y = np.stack([np.clip(2.0 + X[:, 0], 0, 6), 3.0 + 0.5 * X[:, 1] - 0.3 * X[:, 2]], axis=1).astype(np.float32)
    ds = tmp_path / "ds.bin"
    with open(ds, "wb") as f:
        f.write(b"RSVDDS01" + struct.pack("<ii", n, 16) + X.tobytes() + Y.tobytes())
    out = tmp_path / "ctl.bin"
    o = rs.rsvdgb_default_train_opts()
    o.epochs = 150
    o.tau = 0.9
    loss = rs.rsvdgb_controller_train(handle, ds, out, o)
    # loss of the best constant (the label quantiles) for comparison
    tau = 0.9
    base = 0.0
    for c in range(2):
        qv = np.quantile(Y[:, c], tau)
        u = Y[:, c] - qv
        base += np.mean(u * np.where(u < 0, tau - 1, tau))
    assert loss < 0.25 * base, (loss, base)
    raw = open(out, "rb").read()
    assert raw[:8] == b"RSVDMLP1" and struct.unpack("<i", raw[8:12])[0] == 5410
    P = np.frombuffer(raw[12:], dtype="<f4").astype(np.float64)
    gpu = rs.rsvdgb_mlp_forward(handle, dev(P), dev(X[:64])).cpu().numpy()
    assert np.max(np.abs(gpu - oracle.mlp_forward(P, X[:64].astype(np.float64)))) <= 1e-3


@pytest.mark.skipif(not os.path.exists(DEFAULT_CONTROLLER), reason="no trained controller in the package")
def test_trained_controller_gains_over_fixed_q(rs, handle):
    """Held-out planted matrices from the training distribution: the learned
    mode meets the accuracy target (1.05 x the rank-k optimum, + 1e-4 ||A||_F)
    at least as often as fixed p = 10, q = 2, and strictly gains on success
    rate or on passes over A."""
    import torch
    from paper_1608_02148_gb300 import controller_train as ct
    torch.backends.cuda.matmul.allow_tf32 = False
    rs.rsvdgb_controller_load(handle, DEFAULT_CONTROLLER)
    res = ct.evaluate(handle, 16, seed=424242, m=6000, n=2000)
    L, F = res["learned"], res["fixed"]
    assert L["success_rate"] >= F["success_rate"]
    assert L["success_rate"] > F["success_rate"] or L["mean_passes"] < F["mean_passes"], res
