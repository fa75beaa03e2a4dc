"""FP64 CPU oracle for the randomized SVD (arXiv:1608.02148), Python side.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA library.

The arithmetic lives in ``rsvd_oracle.c`` (plain C, double precision, OpenMP);
this module compiles it with gcc into ``oracle/_build/liboracle.so`` and wraps
each exported function with numpy arrays.  See the C file for the paper
passages each function follows.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "rsvd_oracle.c"
_BUILD = _HERE / "_build"
_LIB = _BUILD / "liboracle.so"

SDIST = {"normal": 0, "unif": 1, "rademacher": 2}
DTYPE = {np.dtype(np.float32): 0, np.dtype(np.uint16): 1, np.dtype(np.float64): 2}

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (portable flags: no -march, no FMA contraction)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
               str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(str(_LIB))
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    U64 = ctypes.c_uint64
    lib.oracle_philox4x32_10.argtypes = [P, P, P]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_omega.argtypes = [I64, I64, U64, I, P, I64]
    lib.oracle_omega.restype = None
    lib.oracle_householder_qr.argtypes = [I64, I64, P, P, P]
    lib.oracle_householder_qr.restype = I
    lib.oracle_jacobi_svd.argtypes = [I64, I64, P, P, P, P]
    lib.oracle_jacobi_svd.restype = I
    lib.oracle_rqb.argtypes = [P, I, I64, I64, I64, I, I, I, I, U64, P, P]
    lib.oracle_rqb.restype = I
    lib.oracle_rsvd.argtypes = [P, I, I64, I64, I64, I, I, I, I, U64, P, P, P, P, P]
    lib.oracle_rsvd.restype = I
    lib.oracle_rqb_ex.argtypes = [P, I, I64, I64, I64, I, I, I, I, U64, I, P, P]
    lib.oracle_rqb_ex.restype = I
    lib.oracle_rsvd_ex.argtypes = [P, I, I64, I64, I64, I, I, I, I, U64, I, P, P, P, P, P]
    lib.oracle_rsvd_ex.restype = I
    lib.oracle_lu_pivot.argtypes = [I64, I64, P, P, P, P]
    lib.oracle_lu_pivot.restype = I
    lib.oracle_power_direct.argtypes = [P, I, I64, I64, I64, I64, I, I, U64, P]
    lib.oracle_power_direct.restype = I
    lib.oracle_gemm_ax.argtypes = [P, I, I64, I64, I64, P, I64, P]
    lib.oracle_gemm_ax.restype = I
    lib.oracle_gemm_atx.argtypes = [P, I, I64, I64, I64, P, I64, P]
    lib.oracle_gemm_atx.restype = I
    lib.oracle_residual_fro2.argtypes = [P, I, I64, I64, I64, P, P, P, I64]
    lib.oracle_residual_fro2.restype = ctypes.c_double
    lib.oracle_fro2.argtypes = [P, I, I64, I64, I64]
    lib.oracle_fro2.restype = ctypes.c_double
    lib.oracle_sketch_width.argtypes = [I64, I64, I, I]
    lib.oracle_sketch_width.restype = I64
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = I
    lib.oracle_set_num_threads.argtypes = [I]
    lib.oracle_mlp_params.argtypes = []
    lib.oracle_mlp_params.restype = I
    lib.oracle_mlp_forward.argtypes = [P, P, I64, P]
    lib.oracle_mlp_forward.restype = None
    lib.oracle_mlp_loss_grad.argtypes = [P, P, P, I64, ctypes.c_double, P]
    lib.oracle_mlp_loss_grad.restype = ctypes.c_double
    lib.oracle_set_num_threads.restype = None
    lib.oracle_pqr.argtypes = [I64, I64, P, I64, I, P, P, P, P, P]
    lib.oracle_pqr.restype = I
    lib.oracle_id.argtypes = [I64, I64, P, I64, I, P, P, P]
    lib.oracle_id.restype = I
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _amat(A: np.ndarray):
    """(pointer, dtype code, m, n, lda) of a row-major 2-D array (float32,
    float64, or uint16 holding BF16 bit patterns); rows may be padded."""
    if A.ndim != 2 or A.strides[1] != A.itemsize or A.strides[0] % A.itemsize:
        raise ValueError("A must be 2-D with unit column stride")
    code = DTYPE.get(A.dtype)
    if code is None:
        raise TypeError(f"unsupported dtype {A.dtype}")
    return _ptr(A), code, A.shape[0], A.shape[1], A.strides[0] // A.itemsize


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function on one 128-bit counter and 64-bit key."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def omega(rows: int, l: int, seed: int, sdist: str = "normal") -> np.ndarray:
    """The FP32 test matrix Omega (rows x l) of Sec. 2.3 as defined in rsvd_oracle.c."""
    out = np.zeros((rows, l), dtype=np.float32)
    _load().oracle_omega(rows, l, seed, SDIST[sdist], _ptr(out), l)
    return out


def householder_qr(Y: np.ndarray):
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    m, l = Y.shape
    Q = np.zeros((m, l))
    R = np.zeros((l, l))
    rc = _load().oracle_householder_qr(m, l, _ptr(Y), _ptr(Q), _ptr(R))
    if rc:
        raise RuntimeError(f"householder_qr failed ({rc})")
    return Q, R


def jacobi_svd(M: np.ndarray):
    """One-sided Jacobi: M = Ucols diag(s) J^T, s descending. Returns (Ucols, s, J, sweeps)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    rows, cols = M.shape
    s = np.zeros(cols)
    Uc = np.zeros((rows, cols))
    J = np.zeros((cols, cols))
    sweeps = _load().oracle_jacobi_svd(rows, cols, _ptr(M), _ptr(s), _ptr(Uc), _ptr(J))
    if sweeps < 0:
        raise RuntimeError("jacobi_svd did not converge")
    return Uc, s, J, sweeps


def sketch_width(m: int, n: int, k: int, p: int) -> int:
    return int(_load().oracle_sketch_width(m, n, k, p))


SCHEME = {"qr": 0, "lu": 1}


def lu_pivot(Y: np.ndarray):
    """Pivoted LU of a tall matrix as Algorithm norm_iterations uses it:
    Y = L U, L (m x l) a row permutation of a unit lower trapezoid in Y's row
    order, U (l x l) upper triangular, perm the pivot rows.  Returns (L, U, perm)."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    m, l = Y.shape
    L = np.zeros((m, l))
    U = np.zeros((l, l))
    perm = np.zeros(l, dtype=np.int64)
    rc = _load().oracle_lu_pivot(m, l, _ptr(Y), _ptr(L), _ptr(U), _ptr(perm))
    if rc:
        raise RuntimeError(f"lu_pivot failed ({rc})")
    return L, U, perm


def rqb(A: np.ndarray, k: int, p: int = 10, q: int = 2, sdist: str = "normal", seed: int = 0, scheme: str = "qr"):
    """Algorithm rqb with subspace iterations (scheme "qr", Algorithm
    sub_iterations) or normalized power iterations (scheme "lu", Algorithm
    norm_iterations). For m < n it returns Q, B of the transposed problem."""
    ptr, code, m, n, lda = _amat(A)
    l = sketch_width(m, n, k, p)
    rows, cols = (m, n) if m >= n else (n, m)
    Q = np.zeros((rows, l))
    B = np.zeros((l, cols))
    rc = _load().oracle_rqb_ex(ptr, code, m, n, lda, k, p, q, SDIST[sdist], seed, SCHEME[scheme], _ptr(Q), _ptr(B))
    if rc:
        raise RuntimeError(f"oracle rqb failed ({rc})")
    return Q, B


def rsvd(A: np.ndarray, k: int, p: int = 10, q: int = 2, sdist: str = "normal", seed: int = 0,
         return_qb: bool = False, scheme: str = "qr"):
    """Algorithm rSVD: returns d (k), U (m x k), V (n x k) [, Q, B].  scheme:
    "qr" (subspace iterations) or "lu" (normalized power iterations)."""
    ptr, code, m, n, lda = _amat(A)
    l = sketch_width(m, n, k, p)
    rows, cols = (m, n) if m >= n else (n, m)
    d = np.zeros(k)
    U = np.zeros((m, k))
    V = np.zeros((n, k))
    Q = np.zeros((rows, l)) if return_qb else None
    B = np.zeros((l, cols)) if return_qb else None
    rc = _load().oracle_rsvd_ex(ptr, code, m, n, lda, k, p, q, SDIST[sdist], seed, SCHEME[scheme], _ptr(d), _ptr(U),
                                _ptr(V), _ptr(Q) if return_qb else None, _ptr(B) if return_qb else None)
    if rc:
        raise RuntimeError(f"oracle rsvd failed ({rc})")
    if return_qb:
        return d, U, V, Q, B
    return d, U, V


def values(A: np.ndarray) -> np.ndarray:
    """The stored values of A promoted exactly to float64 (uint16 = BF16 bits)."""
    if A.dtype == np.uint16:
        return (A.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return np.asarray(A, dtype=np.float64)


def rpca(A: np.ndarray, k: int, center: bool = True, scale: bool = True, p: int = 10, q: int = 2,
         sdist: str = "normal", seed: int = 0):
    """Algorithm rpca (Sec. 4.2): principal components of the m x n data
    matrix A (rows = observations, columns = variables).

    Preprocessing of the rpca() interface (Sec. 4.4), written out in FP64:
      centre   mu_j = (1/m) sum_i a_ij                     (center=True, else 0)
      scale    s_j  = sqrt( sum_i (a_ij - mu_j)^2 / (m - 1) )  (scale=True, else 1)
               -- with the centring this is the sample standard deviation, so
               X^T X / (m - 1) is the correlation matrix; without it the root
               mean square with the same m - 1 denominator.  A column with
               s_j = 0 is left as the zero column (its multiplier is 0).
      X = (A - 1 mu^T) diag(1 / s)
    then step 1 [U, Sigma, W] = rsvd(X, k, p, q) (this module's rsvd, the same
    test matrix), step 2 Lambda = Sigma^2 / (m - 1), step 3 Z = U Sigma.
    Returns a dict: rotation W (n x k), eigvals Lambda (k), sdev sqrt(Lambda),
    x Z (m x k), center mu (n), scale s (n)."""
    Av = values(A)
    m, n = Av.shape
    mu = Av.mean(axis=0) if center else np.zeros(n)
    Xc = Av - mu[None, :]
    if scale:
        s = np.sqrt(np.sum(Xc * Xc, axis=0) / (m - 1))
        mult = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    else:
        s = np.ones(n)
        mult = np.ones(n)
    X = np.ascontiguousarray(Xc * mult[None, :])
    d, U, W = rsvd(X, k, p=p, q=q, sdist=sdist, seed=seed)
    lam = d * d / (m - 1)
    return {"rotation": W, "eigvals": lam, "sdev": np.sqrt(lam), "x": U * d[None, :],
            "center": mu, "scale": s, "sigma": d, "X": X}


def pqr(X: np.ndarray, k: int, force_piv=None):
    """QR with column pivoting, k steps (rsvd_oracle.c: oracle_pqr).
    Returns (piv (k,), R (k x cols) in the original column order,
    resid_chosen (k,), resid_max (k,))."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows, cols = X.shape
    piv = np.zeros(k, dtype=np.int64)
    R = np.zeros((k, cols))
    rc_ = np.zeros(k)
    rm_ = np.zeros(k)
    fp = None if force_piv is None else np.ascontiguousarray(force_piv, dtype=np.int64)
    rc = _load().oracle_pqr(rows, cols, _ptr(X), cols, k, _ptr(fp) if fp is not None else None, _ptr(piv), _ptr(R),
                            _ptr(rc_), _ptr(rm_))
    if rc:
        raise RuntimeError(f"oracle pqr failed ({rc})")
    return piv, R, rc_, rm_


def id_decomp(X: np.ndarray, k: int, force_piv=None):
    """Algorithm id: (J (k,), Z (k x cols)) with X ~ X[:, J] Z."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows, cols = X.shape
    J = np.zeros(k, dtype=np.int64)
    Z = np.zeros((k, cols))
    fp = None if force_piv is None else np.ascontiguousarray(force_piv, dtype=np.int64)
    rc = _load().oracle_id(rows, cols, _ptr(X), cols, k, _ptr(fp) if fp is not None else None, _ptr(J), _ptr(Z))
    if rc:
        raise RuntimeError(f"oracle id failed ({rc})")
    return J, Z


def rid(A: np.ndarray, k: int, p: int = 10, q: int = 0, sdist: str = "normal", seed: int = 0, force_piv=None):
    """Algorithm rid (Sec. 7.2): [~, B] = rqb(A, k, p, q); [~, Z, J] = id(B, k);
    C = A(:, J).  Column ID of an m x n A with m >= n (the row ID is the
    column ID of A^T).  Returns (C (m x k), Z (k x n), J (k,), B)."""
    m, n = A.shape
    if m < n:
        raise ValueError("m >= n expected (the row ID is the column ID of A^T)")
    _, B = rqb(A, k, p=p, q=q, sdist=sdist, seed=seed)
    J, Z = id_decomp(B, k, force_piv)
    C = values(A)[:, J]
    return C, Z, J, B


def rcur(A: np.ndarray, k: int, p: int = 10, q: int = 0, sdist: str = "normal", seed: int = 0,
         force_col_piv=None, force_row_piv=None):
    """Algorithm rcur (Sec. 7.1): [C, Z, J] = rid(A, k, p, q);
    [~, S, P] = qr(C^T) pivoted; I = P(1:k); R = A(I, :); U = Z pinv(R)
    (numpy's pseudo-inverse).  Returns (C, U, R, J, I)."""
    C, Z, J, _ = rid(A, k, p=p, q=q, sdist=sdist, seed=seed, force_piv=force_col_piv)
    I, _, _, _ = pqr(np.ascontiguousarray(C.T), k, force_row_piv)
    R = values(A)[I, :]
    U = Z @ np.linalg.pinv(R)
    return C, U, R, J, I


def soft_threshold(X, tau):
    """Elementwise shrinkage sign(x) max(|x| - tau, 0) (Algorithm rrpca
    steps 8 and 10)."""
    return np.sign(X) * np.maximum(np.abs(X) - tau, 0.0)


def predict_rank(d, inv_mu, k, kmax, n_small):
    """Rank prediction of the inexact augmented Lagrange multiplier method
    (the rrpca step 7 the paper delegates to it): svp = number of computed
    singular values above 1/mu; the next target rank is svp + 1 if svp < k,
    else svp + round(0.05 min(m, n)), capped at kmax.  Returns (next k, svp)."""
    svp = int(np.sum(d > inv_mu))
    nk = svp + 1 if svp < k else svp + int(round(0.05 * n_small))
    return max(1, min(nk, kmax)), svp


def rrpca(A: np.ndarray, lam=None, maxiter: int = 50, tol: float = 1e-5, p: int = 10, q: int = 2, k0: int = 2,
          rho: float = 1.5, seed: int = 0, sdist: str = "normal", svd=None):
    """Algorithm rrpca (Sec. 5.2): robust PCA A = L + S by the inexact
    augmented Lagrange multiplier method with a randomized SVD, in FP64.

    Readings where the paper is garbled or silent (following the IALM method
    it cites): mu_0 = 1.25 / ||A||_2 (numpy's 2-norm), multiplier
    Z_0 = A / max(||A||_2, max|a_ij| / lambda), lambda = max(m, n)^(-1/2) by
    default, mu <- min(rho mu, 1e7 mu_0), target rank from predict_rank, stop
    when ||A - L - S||_F <= tol ||A||_F or after maxiter iterations.  Each
    iteration's rSVD uses the test matrix of seed + iteration.  svd (for the
    pins) replaces the randomized SVD by a callable (X, k) -> (d, U, V).
    Returns dict L, S, Z (the last multiplier; Z_0 when maxiter = 0), iters,
    err, k, svp, mu and mu_hist (mu before each iteration, then the last)."""
    M = values(A)
    m, n = M.shape
    ns = min(m, n)
    if lam is None:
        lam = 1.0 / math.sqrt(max(m, n))
    norm2 = float(np.linalg.norm(M, 2))
    mu = 1.25 / norm2
    mu_bar = mu * 1e7
    Z = M / max(norm2, float(np.abs(M).max()) / lam)
    S = np.zeros_like(M)
    L = np.zeros_like(M)
    normM = float(np.linalg.norm(M))
    kmax = min(ns - 1, 224 - p)
    k = min(k0, kmax)
    err = float("inf")
    svp = 0
    it = 0
    mu_hist = [mu]
    for it in range(1, maxiter + 1):
        X = np.ascontiguousarray(M - S + Z / mu)
        if svd is None:
            d, U, V = rsvd(X, k, p=p, q=q, sdist=sdist, seed=seed + it)
        else:
            d, U, V = svd(X, k)
        k_next, svp = predict_rank(d, 1.0 / mu, k, kmax, ns)
        ds = np.maximum(d[:svp] - 1.0 / mu, 0.0)
        L = (U[:, :svp] * ds[None, :]) @ V[:, :svp].T
        S = soft_threshold(M - L + Z / mu, lam / mu)
        R = M - L - S
        Z = Z + mu * R
        mu = min(rho * mu, mu_bar)
        mu_hist.append(mu)
        err = float(np.linalg.norm(R)) / normM
        k = k_next
        if err < tol:
            break
    return {"L": L, "S": S, "Z": Z, "iters": it, "err": err, "k": k, "svp": svp, "mu": mu, "mu_hist": mu_hist}


def power_direct(A: np.ndarray, l: int, q: int, sdist: str = "normal", seed: int = 0) -> np.ndarray:
    """Algorithm poweriter_direct: Y = (A A^T)^q A Omega (m >= n)."""
    ptr, code, m, n, lda = _amat(A)
    Y = np.zeros((m, l))
    rc = _load().oracle_power_direct(ptr, code, m, n, lda, l, q, SDIST[sdist], seed, _ptr(Y))
    if rc:
        raise RuntimeError(f"oracle power_direct failed ({rc})")
    return Y


def gemm_ax(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    ptr, code, m, n, lda = _amat(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    assert X.shape[0] == n
    Y = np.zeros((m, X.shape[1]))
    _load().oracle_gemm_ax(ptr, code, m, n, lda, _ptr(X), X.shape[1], _ptr(Y))
    return Y


def gemm_atx(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    ptr, code, m, n, lda = _amat(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    assert X.shape[0] == m
    Z = np.zeros((n, X.shape[1]))
    _load().oracle_gemm_atx(ptr, code, m, n, lda, _ptr(X), X.shape[1], _ptr(Z))
    return Z


def residual_fro2(A: np.ndarray, U: np.ndarray, d: np.ndarray, V: np.ndarray) -> float:
    ptr, code, m, n, lda = _amat(A)
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    k = d.shape[0]
    return float(_load().oracle_residual_fro2(ptr, code, m, n, lda, _ptr(U), _ptr(d), _ptr(V), k))


def fro2(A: np.ndarray) -> float:
    ptr, code, m, n, lda = _amat(A)
    return float(_load().oracle_fro2(ptr, code, m, n, lda))


def canonical_signs(U: np.ndarray, V: np.ndarray):
    """Flip each singular pair (u_i, v_i) so that the largest-magnitude entry
    of v_i is positive (ties: lowest index).  Singular vectors are unique only
    up to such a sign."""
    U = U.copy()
    V = V.copy()
    for c in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, c])))
        if V[i, c] < 0:
            U[:, c] = -U[:, c]
            V[:, c] = -V[:, c]
    return U, V


# ---------------------------------------------------------------- controller network (FP64)
def mlp_params() -> int:
    return _load().oracle_mlp_params()


def mlp_forward(P, X):
    """Network outputs (n x 2) for float64 parameters P and inputs X (n x 16)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros((X.shape[0], 2))
    _load().oracle_mlp_forward(_ptr(P), _ptr(X), X.shape[0], _ptr(out))
    return out


def mlp_loss_grad(P, X, Y, tau=0.9, with_grad=True):
    """Mean pinball loss and its gradient w.r.t. the trainable parameters."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    g = np.zeros(mlp_params() - 32) if with_grad else None
    loss = _load().oracle_mlp_loss_grad(_ptr(P), _ptr(X), _ptr(Y), X.shape[0], float(tau),
                                       _ptr(g) if with_grad else None)
    return loss, g


def controller_features(A: np.ndarray, k: int, p_max: int = 40, seed: int = 0, sdist: str = "normal"):
    """The 16 controller features of a row-major A with m >= n, as the library
    defines them: the sketch Y = A Omega with l = min(k + p_max, n) columns
    (the test matrix of Sec. 2.3), the diagonal r_j = |R_jj| of its QR factor
    (Householder, FP64; unique up to signs) and ||A||_F^2; then
      [log10 m, log10 n, log10 k, k / n,
       log10(r_j / r_1) for j = ceil(k/4), ceil(k/2), ceil(3k/4), k, k + 1,
                            k + max(p_max // 4, 1), k + max(p_max // 2, 1), l
                        (indices clamped to [1, l]),
       sum_{j<=k} r_j^2 / sum_j r_j^2,
       log10(||Y||_F^2 / (l ||A||_F^2)),
       log10(r_k / r_l),
       p_max / k]."""
    m, n = A.shape
    if m < n:
        raise ValueError("m >= n expected")
    l = min(k + p_max, n)
    Om = omega(n, l, seed, sdist).astype(np.float64)
    Y = gemm_ax(A, Om)
    _, R = householder_qr(Y)
    r = np.maximum(np.abs(np.diag(R)), 1e-30)
    fa = fro2(A)

    def lr(j):
        j = min(max(j, 1), l)
        return math.log10(r[j - 1] / r[0])

    e_all = float(np.sum(r ** 2))
    e_k = float(np.sum(r[:k] ** 2))
    tr = float(np.sum(Y * Y))
    f = [math.log10(m), math.log10(n), math.log10(k), k / n,
         lr((k + 3) // 4), lr((k + 1) // 2), lr((3 * k + 3) // 4), lr(k), lr(k + 1),
         lr(k + max(p_max // 4, 1)), lr(k + max(p_max // 2, 1)), lr(l),
         e_k / e_all if e_all > 0 else 1.0,
         math.log10(tr / (l * fa)) if (fa > 0 and tr > 0) else 0.0,
         math.log10(r[min(k, l) - 1] / r[l - 1]),
         p_max / k]
    return np.array(f)
