"""Pins of the oracle's controller network (CPU only).

The network is not from the paper (which leaves q and p to the user,
Sec. 3.4); its definition is the library's parameter format.  The oracle's
forward pass and reverse-mode gradient are pinned here by things other than
themselves: central finite differences, a hand-built network with a known
output, and the closed form of a network whose output is its bias.
"""
import math

import numpy as np
import pytest

import oracle

NP = 5410
NT = NP - 32


def random_params(rng, scale=0.3):
    P = rng.standard_normal(NP) * scale
    P[:16] = rng.standard_normal(16) * 0.1  # mu
    P[16:32] = np.abs(rng.standard_normal(16)) + 0.5  # sd > 0
    return P


def test_parameter_count_matches_the_format():
    assert oracle.mlp_params() == NP == 2 * 16 + 64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2


@pytest.mark.parametrize("tau", [0.9, 0.5, 0.1])
def test_gradient_matches_central_differences(tau):
    rng = np.random.default_rng(3)
    P = random_params(rng)
    X = rng.standard_normal((9, 16))
    Y = rng.standard_normal((9, 2)) * 2
    loss, g = oracle.mlp_loss_grad(P, X, Y, tau)
    # every block of the parameter vector: W1, b1, W2, b2, W3, b3
    blocks = [(0, 1024), (1024, 1088), (1088, 5184), (5184, 5248), (5248, 5376), (5376, 5378)]
    eps = 1e-6
    for lo, hi in blocks:
        for e in rng.choice(np.arange(lo, hi), size=min(12, hi - lo), replace=False):
            Pp = P.copy()
            Pp[32 + e] += eps
            Pm = P.copy()
            Pm[32 + e] -= eps
            num = (oracle.mlp_loss_grad(Pp, X, Y, tau, False)[0] - oracle.mlp_loss_grad(Pm, X, Y, tau, False)[0]) / (
                2 * eps)
            assert abs(num - g[e]) <= 1e-6 * max(1.0, abs(num)), (lo, e, num, g[e])


def test_bias_only_network_has_the_closed_form_loss_and_gradient():
    """W3 = 0: the output is b3, the loss is the mean pinball loss of y - b3,
    d/db3 = -mean(tau - [u < 0]) and every other gradient vanishes."""
    rng = np.random.default_rng(5)
    P = random_params(rng)
    P[32 + 5248:32 + 5376] = 0.0  # W3
    b3 = np.array([0.7, -0.2])
    P[32 + 5376:] = b3
    X = rng.standard_normal((11, 16))
    Y = rng.standard_normal((11, 2))
    tau = 0.9
    loss, g = oracle.mlp_loss_grad(P, X, Y, tau)
    U = Y - b3[None, :]
    W = np.where(U < 0, tau - 1.0, tau)
    assert abs(loss - np.mean(np.sum(U * W, axis=1))) < 1e-14
    assert np.allclose(g[5376:], -np.mean(W, axis=0), atol=1e-15)
    assert np.all(g[:5248] == 0.0)


def test_hand_built_network_computes_abs_and_a_sum():
    """h1 = relu(+-x_0) (units 0, 1), h2 copies them, o_0 = h2_0 + h2_1 = |x_0|
    and o_1 = relu(x_1) + 3 through unit 2: checks the wiring of every layer and
    the standardisation."""
    P = np.zeros(NP)
    mu = np.zeros(16)
    mu[1] = 1.0
    sd = np.ones(16)
    sd[0] = 2.0
    P[:16], P[16:32] = mu, sd
    W1 = np.zeros((64, 16))
    W1[0, 0], W1[1, 0], W1[2, 1] = 1.0, -1.0, 1.0
    W2 = np.zeros((64, 64))
    W2[0, 0] = W2[1, 1] = W2[2, 2] = 1.0
    W3 = np.zeros((2, 64))
    W3[0, 0] = W3[0, 1] = 1.0
    W3[1, 2] = 1.0
    P[32:32 + 1024] = W1.ravel()
    P[32 + 1088:32 + 5184] = W2.ravel()
    P[32 + 5248:32 + 5376] = W3.ravel()
    P[32 + 5376:] = [0.0, 3.0]
    rng = np.random.default_rng(1)
    X = rng.standard_normal((20, 16)) * 3
    out = oracle.mlp_forward(P, X)
    assert np.allclose(out[:, 0], np.abs(X[:, 0] / 2.0), atol=1e-15)
    assert np.allclose(out[:, 1], np.maximum(X[:, 1] - 1.0, 0.0) + 3.0, atol=1e-15)


def test_features_of_an_exact_low_rank_matrix():
    """Rank-r A (r < k): the sketch spans col(A) exactly, so all of its energy
    sits in the top r <= k singular values (energy fraction 1) and
    sum s_i^2 / (l ||A||_F^2) is the mean squared norm of the l sketch
    columns relative to ||A||_F^2, ~1 for Gaussian columns (E ||A w||^2 =
    ||A||_F^2)."""
    rng = np.random.default_rng(9)
    m, n, r, k = 300, 120, 6, 10
    A = (rng.standard_normal((m, r)) @ rng.standard_normal((r, n))).astype(np.float32)
    f = oracle.controller_features(A, k, p_max=20, seed=4)
    assert f.shape == (16,)
    assert abs(f[0] - math.log10(m)) < 1e-12 and abs(f[2] - math.log10(k)) < 1e-12
    assert abs(f[1] - math.log10(n)) < 1e-12 and abs(f[3] - k / n) < 1e-12 and abs(f[15] - 20 / k) < 1e-12
    assert abs(f[12] - 1.0) < 1e-12
    assert abs(f[13]) < 0.3
    assert f[11] < -6  # r_l / r_1 at the FP32 storage level of A: rank r < l


@pytest.mark.parametrize("r", [1, 3, 4, 5, 7, 8, 9, 12, 13, 17, 18, 27])
def test_decay_features_sit_at_their_indices(r):
    """The QR factor of a sketch of rank r has R_jj = 0 (to rounding) exactly
    for j > r, so log10(r_j / r_1) is ordinary for j <= r and far below for
    j > r.  With k = 8, p_max = 20 (l = 28) the decay features read the
    indices ceil(k/4), ceil(k/2), ceil(3k/4), k, k + 1, k + p_max/4,
    k + p_max/2 and l = 2, 4, 6, 8, 9, 13, 18, 28; sweeping r across them
    fixes each index (an index off by one moves a feature across a rank
    boundary)."""
    rng = np.random.default_rng(100 + r)
    m, n, k = 200, 60, 8
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    f = oracle.controller_features(A, k, p_max=20, seed=6)
    for t, j in zip(range(4, 12), (2, 4, 6, 8, 9, 13, 18, 28)):
        if j <= r:
            assert f[t] > -4, (t, j, f[t])
        else:
            assert f[t] < -10, (t, j, f[t])
    if k <= r < 28:  # log10(r_k / r_l): r_k ordinary, r_l beyond the rank
        assert f[14] > 10, f[14]
    # energy of the first k diagonal entries: all of it iff the rank is <= k
    if r <= k:
        assert abs(f[12] - 1.0) < 1e-12, f[12]
    else:
        assert f[12] < 1.0 - 1e-6, f[12]
