"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random matrices with a planted spectrum.  It holds none
of the randomized-SVD arithmetic: orthonormal factors come from a library QR
(numpy QR on the host; device matmuls with a host Cholesky), never from this project's kernels or
from its CPU oracle.  Both the CUDA path and the oracle are fed the same stored
values produced here.

Recipes (all seeds explicit):

* ``planted(m, n, sigma)`` -- A = U diag(sigma) V^T with U (m x r) and V (n x r)
  the Q factors of seeded N(0,1) matrices, r = len(sigma); formed in float64
  and stored as float32 (or BF16).  With sigma_i = exp(-i/20) on 2000 x 1000
  this is the small planted workload; truncating sigma plants an exact rank.
* ``spiked_noise(m, n, sigma, noise_std)`` -- A = W_m diag(sigma) W_n^T + E
  with E i.i.d. N(0, noise_std^2): the 200000 x 2000 workload uses
  sigma_i = 1/i and noise_std = 1e-3.  Built with torch on any device.
* ``ragged_batch(...)`` -- many small planted matrices with log-uniform shapes
  and exponential spectra exp(-r i), r uniform.
"""
from __future__ import annotations

import math

import numpy as np


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 values to BF16 (round to nearest even) and return the
    16-bit patterns as uint16."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def _orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    # Fix the column signs so the factor is a deterministic function of the seed.
    return q * np.sign(np.diag(r))[None, :]


def planted(m: int, n: int, sigma, seed: int, dtype=np.float32) -> np.ndarray:
    """A = U diag(sigma) V^T (float64 product, stored in ``dtype``)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    assert r <= min(m, n)
    rng = np.random.default_rng(seed)
    U = _orthonormal(rng, m, r)
    V = _orthonormal(rng, n, r)
    A = (U * sigma[None, :]) @ V.T
    if dtype == "bf16":
        return bf16_bits(A.astype(np.float32))
    return A.astype(dtype)


def exp_spectrum(count: int, rate: float) -> np.ndarray:
    """sigma_i = exp(-rate * i), i = 1..count."""
    return np.exp(-rate * np.arange(1, count + 1, dtype=np.float64))


def small_planted(seed: int = 0x160802148 + 1000) -> np.ndarray:
    """2000 x 1000, sigma_i = exp(-i/20) (the small planted workload)."""
    return planted(2000, 1000, exp_spectrum(1000, 1.0 / 20.0), seed)


def _orthonormal_torch(G):
    """Orthonormalise the columns of a tall torch matrix with device matmuls
    (FP64 Gram) and a host (numpy, float64) factorisation of the small Gram
    matrix, twice.
    Only library products are used; torch's device linear-algebra module is
    not needed."""
    import torch

    for _ in range(2):
        Gd = G.double()
        gram = (Gd.T @ Gd).cpu().numpy()  # FP64 Gram: a square Gaussian has kappa ~ n
        del Gd
        R = np.linalg.cholesky(gram).T
        Rinv = np.linalg.inv(R)
        G = G @ torch.as_tensor(Rinv, dtype=G.dtype, device=G.device)
    return G


def spiked_noise(m: int, n: int, sigma, noise_std: float, seed: int, device="cpu", dtype=None):
    """A = W_m diag(sigma) W_n^T + E on a torch device (float32 storage).

    W_m (m x r) and W_n (n x r) are seeded Gaussians orthonormalised with
    library products (device matmul, host Cholesky),
    r = len(sigma); E is i.i.d. N(0, noise_std^2)."""
    import torch

    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float32), device=dev)
    r = sig.shape[0]
    Wm = _orthonormal_torch(torch.randn(m, r, generator=gen, device=dev, dtype=torch.float32))
    Wn = _orthonormal_torch(torch.randn(n, r, generator=gen, device=dev, dtype=torch.float32))
    A = torch.randn(m, n, generator=gen, device=dev, dtype=torch.float32)
    A.mul_(noise_std)
    A.addmm_(Wm * sig[None, :], Wn.T)
    del Wm, Wn
    if dtype is not None:
        A = A.to(dtype)
    return A


def ragged_shapes(count: int, m_range, n_range, seed: int):
    """Log-uniform integer shapes (m_b, n_b) and exponential decay rates."""
    rng = np.random.default_rng(seed)
    lm = rng.uniform(math.log(m_range[0]), math.log(m_range[1]), count)
    ln = rng.uniform(math.log(n_range[0]), math.log(n_range[1]), count)
    ms = np.rint(np.exp(lm)).astype(np.int64)
    ns = np.rint(np.exp(ln)).astype(np.int64)
    rates = rng.uniform(0.05, 0.5, count)
    return ms, ns, rates


def ragged_batch(count: int, m_range=(256, 4096), n_range=(64, 1024), seed: int = 0, device="cpu",
                 shapes=None):
    """Many matrices A_b = H_U S_b H_V with an exponential spectrum
    sigma_i = exp(-r_b i) (r_b uniform in [0.05, 0.5]) and log-uniform shapes.

    S_b holds sigma on a random partial permutation; H_U, H_V are products of
    two random Householder reflectors, so A_b has exactly the planted singular
    values (rotational invariance of the Gaussian sketch makes the choice of
    orthogonal factors immaterial).  Built with torch on any device; returns
    (list of float32 tensors, decay rates)."""
    import torch

    if shapes is None:
        ms, ns, rates = ragged_shapes(count, m_range, n_range, seed)
    else:
        ms, ns, rates = shapes
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    mats = []
    for m, n, r in zip(ms.tolist(), ns.tolist(), rates.tolist()):
        mn = min(m, n)
        sig = torch.exp(-r * torch.arange(1, mn + 1, dtype=torch.float64, device=device))
        pm = torch.randperm(m, generator=gen, device=device)[:mn]
        pn = torch.randperm(n, generator=gen, device=device)[:mn]
        A = torch.zeros(m, n, dtype=torch.float64, device=device)
        A[pm, pn] = sig
        for _ in range(2):
            u = torch.randn(m, 1, generator=gen, device=device, dtype=torch.float64)
            u /= u.norm()
            A -= 2.0 * u @ (u.T @ A)
            v = torch.randn(n, 1, generator=gen, device=device, dtype=torch.float64)
            v /= v.norm()
            A -= 2.0 * (A @ v) @ v.T
        mats.append(A.to(torch.float32).contiguous())
    return mats, rates


def planted_reflector(m: int, n: int, sigma, seed: int, device="cpu"):
    """A = H_U diag(sigma) H_V (float32), sigma on the leading diagonal and H_U,
    H_V products of two seeded Householder reflectors: exactly the planted
    singular values, built in FP64 on the device."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    mn = min(m, n)
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64)[:mn], device=device)
    A = torch.zeros(m, n, dtype=torch.float64, device=device)
    idx = torch.arange(sig.shape[0], device=device)
    A[idx, idx] = sig
    for _ in range(2):
        u = torch.randn(m, 1, generator=gen, device=device, dtype=torch.float64)
        u /= u.norm()
        A -= 2.0 * u @ (u.T @ A)
        v = torch.randn(n, 1, generator=gen, device=device, dtype=torch.float64)
        v /= v.norm()
        A -= 2.0 * (A @ v) @ v.T
    return A.to(torch.float32).contiguous()


def step_noise(m: int, n: int, step: int, noise_std: float, seed: int, device="cpu", bf16: bool = True):
    """Step spectrum (sigma = 1 for i <= step, 1e-2 beyond) on two-reflector
    orthogonal factors (planted_reflector) plus i.i.d. N(0, noise_std^2)
    noise added in row blocks, stored BF16 (or float32)."""
    import torch

    sigma = np.where(np.arange(1, min(m, n) + 1) <= step, 1.0, 1e-2)
    A = planted_reflector(m, n, sigma, seed, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    for r0 in range(0, m, 8192):
        blk = A[r0:r0 + 8192]
        blk.add_(torch.randn(blk.shape, generator=gen, device=device, dtype=torch.float32), alpha=noise_std)
    return A.to(torch.bfloat16) if bf16 else A


def controller_spectrum(rng, k: int, count: int):
    """A random spectrum of one of three families (descending, sigma_1 = 1):
    exponential exp(-r (i - 1)), r log-uniform in [1e-3, 0.5]; power law
    i^-alpha, alpha uniform in [0.25, 3]; step: 1 for i <= s, s uniform in
    [k/2, 2k], then delta log-uniform in [1e-4, 0.3].  Returns (sigma, label)."""
    i = np.arange(1, count + 1, dtype=np.float64)
    kind = int(rng.integers(0, 3))
    if kind == 0:
        r = math.exp(rng.uniform(math.log(1e-3), math.log(0.5)))
        return np.exp(-r * (i - 1)), f"exp r={r:.4g}"
    if kind == 1:
        a = rng.uniform(0.25, 3.0)
        return i ** (-a), f"power alpha={a:.3g}"
    s = int(rng.integers(max(1, k // 2), 2 * k + 1))
    d = math.exp(rng.uniform(math.log(1e-4), math.log(0.3)))
    return np.where(i <= s, 1.0, d), f"step s={s} delta={d:.3g}"


def pca_data(m: int, n: int, rank: int, seed: int, decay: float = 0.85, noise_std: float = 0.05,
             mean_ratio: float = 5.0, scale_range=(0.1, 10.0), device="cpu", zero_var_cols=0):
    """Observations x variables data with heterogeneous units, as the PCA
    examples treat them (rows = observations, columns = variables):

        A = (F L^T + E) diag(c) + 1 mu^T

    F (m x rank) i.i.d. N(0, 1) latent factors; L (n x rank) i.i.d. N(0, 1)
    loadings with column j scaled by decay^j (a decaying spectrum of the
    correlation matrix); E i.i.d. N(0, noise_std^2); c log-uniform in
    scale_range (units); mu_j = mean_ratio * c_j * N(0, 1) (column offsets
    several spreads away from zero).  The last ``zero_var_cols`` columns are
    constant (zero variance).  float32 storage, built with torch on any device."""
    import torch

    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    F = torch.randn(m, rank, generator=gen, device=dev, dtype=torch.float32)
    L = torch.randn(n, rank, generator=gen, device=dev, dtype=torch.float32)
    L *= decay ** torch.arange(rank, device=dev, dtype=torch.float32)[None, :]
    A = torch.randn(m, n, generator=gen, device=dev, dtype=torch.float32)
    A.mul_(noise_std)
    A.addmm_(F, L.T)
    del F, L
    lo, hi = math.log(scale_range[0]), math.log(scale_range[1])
    c = torch.exp(lo + (hi - lo) * torch.rand(n, generator=gen, device=dev, dtype=torch.float32))
    mu = mean_ratio * c * torch.randn(n, generator=gen, device=dev, dtype=torch.float32)
    A.mul_(c[None, :]).add_(mu[None, :])
    if zero_var_cols > 0:
        A[:, n - zero_var_cols:] = mu[None, n - zero_var_cols:]
    return A.contiguous()


def low_rank_plus_sparse(m: int, n: int, rank: int, density: float, seed: int, magnitude: float = 1.0):
    """A = L0 + S0 for robust PCA: L0 = F G^T / sqrt(rank) with F (m x rank)
    and G (n x rank) i.i.d. N(0, 1), so the entries of L0 are N(0, 1); S0
    holds gross corruptions on a random fraction `density` of the entries,
    uniform in [-5 magnitude, 5 magnitude], zero elsewhere.  float64 numpy
    (L0, S0, A).  The robust-PCA example of Sec. 5 (a 300 x 300 rank-5
    matrix with 20 % corrupted entries) is low_rank_plus_sparse(300, 300, 5, 0.2, seed)."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((m, rank))
    G = rng.standard_normal((n, rank))
    L0 = F @ G.T / math.sqrt(rank)
    mask = rng.random((m, n)) < density
    S0 = np.where(mask, rng.uniform(-5.0 * magnitude, 5.0 * magnitude, (m, n)), 0.0)
    return L0, S0, L0 + S0


def rrpca_example(seed: int, m: int = 300, n: int = 300, rank: int = 5, density: float = 0.2):
    """The robust-PCA simulation of Sec. 5.5: L = L1 L2 with L1 (m x rank) and
    L2 (rank x n) i.i.d. N(0, 1); S i.i.d. uniform on [-500, 500] kept with
    probability 0.2 (Bernoulli mask); A = L + S.  float64 numpy (L, S, A)."""
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    S = rng.uniform(-500.0, 500.0, (m, n)) * (rng.random((m, n)) < density)
    return L, S, L + S
