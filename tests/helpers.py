"""Comparison helpers shared by the parity tests (no method arithmetic)."""
import math

import numpy as np

U32 = 2.0 ** -24  # unit roundoff of FP32


def sin_theta(A, B):
    """Sine of the largest principal angle between span(A) and span(B)."""
    Qa, _ = np.linalg.qr(np.asarray(A, dtype=np.float64))
    Qb, _ = np.linalg.qr(np.asarray(B, dtype=np.float64))
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))


def subspace_tol(sig_all, k, norm2, base=1e-4):
    """FP32 subspace tolerance with the gap rule: max(base, 10 u32 ||A||_2 / gap_k)
    where gap_k = sigma_k - sigma_{k+1} of the reference spectrum."""
    if k >= len(sig_all):
        return base
    gap = sig_all[k - 1] - sig_all[k]
    if gap <= 0:
        return 1.0
    return max(base, 10 * U32 * norm2 / gap)


def sigma_err(d_gpu, d_ref):
    d_gpu = np.asarray(d_gpu, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    return float(np.max(np.abs(d_gpu - d_ref)) / d_ref[0])


def ulp_distance_f32(a, b):
    """Distance in units in the last place between float32 arrays."""
    ai = np.asarray(a, dtype=np.float32).view(np.int32).astype(np.int64)
    bi = np.asarray(b, dtype=np.float32).view(np.int32).astype(np.int64)
    ai = np.where(ai < 0, -(ai & 0x7FFFFFFF), ai)
    bi = np.where(bi < 0, -(bi & 0x7FFFFFFF), bi)
    return np.abs(ai - bi)
