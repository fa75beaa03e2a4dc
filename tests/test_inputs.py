"""The seeded input generators produce the workloads they state (CPU only):
planted spectra are exact, shapes and rates fall in their ranges, the noise,
sparsity and unit recipes hold.  The generators hold none of the method's
arithmetic; these checks use numpy / torch library routines."""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_1608_02148_gb300 import inputs


def test_bf16_rounding_matches_torch():
    """Round to nearest even, as torch's float32 -> bfloat16 conversion."""
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 1e3,
                        np.array([0.0, -0.0, np.inf, -np.inf, 1e-40, -3e-39, 3.4e38], dtype=np.float32)])
    # exact ties: low 16 bits 0x8000 with even and odd kept parts
    ties = (np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40490000 | 0x8000], dtype=np.uint32)).view(np.float32)
    a = np.concatenate([a, ties])
    mine = inputs.bf16_bits(a)
    ref = torch.from_numpy(a).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(mine, ref)
    np.testing.assert_array_equal(inputs.bf16_to_f32(mine), torch.from_numpy(a).to(torch.bfloat16).float().numpy())


def test_planted_has_exactly_the_planted_spectrum():
    sigma = inputs.exp_spectrum(40, 0.1)
    A = inputs.planted(120, 60, sigma, seed=3, dtype=np.float64)
    s = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(s[:40], sigma, rtol=1e-12, atol=1e-14)
    assert np.all(s[40:] < 1e-13)
    A32 = inputs.planted(120, 60, sigma, seed=3)
    assert A32.dtype == np.float32
    np.testing.assert_allclose(A32, A, atol=1e-7 * np.abs(A).max())
    np.testing.assert_array_equal(A32, inputs.planted(120, 60, sigma, seed=3))  # a function of the seed
    assert not np.array_equal(A32, inputs.planted(120, 60, sigma, seed=4))


def test_small_planted_workload_recipe():
    """2000 x 1000, sigma_i = exp(-i/20), i = 1..1000."""
    A = inputs.small_planted()
    assert A.shape == (2000, 1000) and A.dtype == np.float32
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(s[:50], np.exp(-np.arange(1, 51) / 20.0), rtol=1e-5)


def test_spiked_noise_recipe():
    """A = W_m diag(sigma) W_n^T + E: the spikes well above the noise edge
    come out at about sqrt(sigma^2 + s^2 (m + n)) and the energy is
    sum sigma^2 + s^2 m n."""
    m, n, s_noise = 3000, 200, 1e-3
    sigma = 1.0 / np.arange(1, n + 1)
    A = inputs.spiked_noise(m, n, sigma, s_noise, seed=5).double().numpy()
    sv = np.linalg.svd(A, compute_uv=False)
    expect = np.sqrt(sigma[:3] ** 2 + s_noise ** 2 * (m + n))
    np.testing.assert_allclose(sv[:3], expect, rtol=1e-2)
    energy = np.sum(sigma ** 2) + s_noise ** 2 * m * n
    assert abs(np.sum(A * A) / energy - 1.0) < 2e-2
    edge = s_noise * (math.sqrt(m) + math.sqrt(n))
    assert sv[-1] < edge  # the bulk sits at the noise level


def test_step_noise_recipe():
    """The BF16-stored step-spectrum workload: sigma = 1 for i <= step and
    1e-2 beyond on the two-reflector factors, plus i.i.d. N(0, s^2) noise;
    the BF16 form is the FP32 form rounded to BF16."""
    m, n, step, s_noise = 2000, 600, 40, 1e-5
    A32 = inputs.step_noise(m, n, step, s_noise, seed=9, bf16=False)
    A16 = inputs.step_noise(m, n, step, s_noise, seed=9, bf16=True)
    assert A32.dtype == torch.float32 and A16.dtype == torch.bfloat16
    assert torch.equal(A16, A32.to(torch.bfloat16))
    sigma = np.where(np.arange(1, n + 1) <= step, 1.0, 1e-2)
    sv = np.linalg.svd(A32.double().numpy(), compute_uv=False)
    E = (A32.double() - inputs.planted_reflector(m, n, sigma, seed=9).double()).numpy()
    assert abs(E.std() / s_noise - 1.0) < 2e-2 and abs(E.mean()) < 0.1 * s_noise
    # the noise's spectral norm is the Gaussian edge s (sqrt m + sqrt n), and by
    # Weyl's inequality every singular value stays within it of the planted one
    e2 = np.linalg.norm(E, 2)
    assert abs(e2 / (s_noise * (math.sqrt(m) + math.sqrt(n))) - 1.0) < 5e-2
    assert np.all(np.abs(sv - sigma) <= e2 + 1e-6)
    assert np.all(sv[:step] > 0.99) and np.all(np.abs(sv[step:] - 1e-2) < 1e-3)
    energy = np.sum(sigma ** 2) + s_noise ** 2 * m * n
    assert abs(float((A32.double() ** 2).sum()) / energy - 1.0) < 1e-3


def test_ragged_shapes_and_rates_in_range():
    ms, ns, rates = inputs.ragged_shapes(4096, (256, 4096), (64, 1024), seed=0x160802148 + 4000)
    assert ms.min() >= 256 and ms.max() <= 4096 and ns.min() >= 64 and ns.max() <= 1024
    assert rates.min() >= 0.05 and rates.max() <= 0.5
    # log-uniform: the mean of log m sits mid-range (standard error ~ 0.8 / sqrt(4096))
    assert abs(np.mean(np.log(ms)) - 0.5 * (math.log(256) + math.log(4096))) < 0.05
    assert abs(np.mean(np.log(ns)) - 0.5 * (math.log(64) + math.log(1024))) < 0.05
    assert 0.08 < np.mean(ms < ns) < 0.18  # about one matrix in eight is wide


def test_ragged_batch_and_reflector_matrices_have_the_planted_spectrum():
    ms = np.array([300, 90, 257]); ns = np.array([70, 200, 129]); rates = np.array([0.05, 0.3, 0.5])
    mats, r = inputs.ragged_batch(3, seed=9, shapes=(ms, ns, rates))
    for A, m, n, rate in zip(mats, ms, ns, rates):
        assert tuple(A.shape) == (m, n) and A.dtype == torch.float32
        s = np.linalg.svd(A.double().numpy(), compute_uv=False)
        np.testing.assert_allclose(s, np.exp(-rate * np.arange(1, min(m, n) + 1)), rtol=2e-5, atol=1e-7)
    B = inputs.planted_reflector(150, 80, inputs.exp_spectrum(80, 0.1), seed=2)
    s = np.linalg.svd(B.double().numpy(), compute_uv=False)
    np.testing.assert_allclose(s, inputs.exp_spectrum(80, 0.1), rtol=2e-5, atol=1e-7)


def test_controller_spectra_families():
    rng = np.random.default_rng(0)
    seen = set()
    for _ in range(60):
        sig, label = inputs.controller_spectrum(rng, 40, 300)
        assert sig[0] == 1.0 and np.all(np.diff(sig) <= 0) and sig[-1] > 0
        kind = label.split()[0]
        seen.add(kind)
        val = float(label.split("=")[1].split()[0])
        if kind == "exp":
            assert 1e-3 <= val <= 0.5
        elif kind == "power":
            assert 0.25 <= val <= 3.0
        else:
            assert 20 <= val <= 80
    assert seen == {"exp", "power", "step"}


def test_pca_data_recipe():
    """Offsets several spreads from zero, units spanning two decades, a
    dominant rank-r structure in the correlation matrix, constant columns."""
    m, n, r = 4000, 120, 10
    A = inputs.pca_data(m, n, r, seed=3, zero_var_cols=2).double().numpy()
    sd = A.std(axis=0, ddof=1)
    assert np.all(sd[-2:] == 0) and np.all(sd[:-2] > 0)
    mean = A.mean(axis=0)
    assert np.median(np.abs(mean[:-2]) / sd[:-2]) > 1.0
    assert sd[:-2].max() / sd[:-2].min() > 10
    ev = np.linalg.eigvalsh(np.corrcoef(A[:, :-2].T))[::-1]
    assert ev[:r].sum() / ev.sum() > 0.9


def test_low_rank_plus_sparse_recipe():
    L0, S0, A = inputs.low_rank_plus_sparse(200, 150, 4, 0.1, seed=1)
    assert np.linalg.matrix_rank(L0) == 4
    assert abs(np.mean(S0 != 0) - 0.1) < 0.01 and np.abs(S0).max() <= 5.0
    assert abs(L0.std() - 1.0) < 0.1
    np.testing.assert_array_equal(A, L0 + S0)


def test_rrpca_example_is_the_papers_simulation():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))["rrpca_example"]
    m, n = gold["shape"]
    L, S, A = inputs.rrpca_example(1, m, n, gold["rank"], gold["sparse_fraction"])
    assert L.shape == (m, n) and np.linalg.matrix_rank(L) == gold["rank"]
    lo, hi = gold["sparse_range"]
    assert S.min() >= lo and S.max() <= hi
    assert abs(np.mean(S != 0) - gold["sparse_fraction"]) < 0.01
    np.testing.assert_array_equal(A, L + S)
