"""Python binding of librsvdgb (ctypes): argument marshalling only.

Every function here forwards torch tensors' device pointers and sizes to the
C entry point of the same name declared in include/rsvdgb.h; all arithmetic
runs in the library's CUDA kernels.  PyTorch supplies device memory and the
current CUDA stream.  If the shared library has not been built, loading fails
with an error -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "librsvdgb.so"

RSVDGB_OK = 0
RSVDGB_ERR_INVALID_ARG = 1
STATUS = {0: "OK", 1: "ERR_INVALID_ARG", 2: "ERR_NOMEM", 3: "ERR_CUDA", 4: "ERR_BREAKDOWN", 5: "ERR_NONFINITE",
          6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}
F32, BF16 = 0, 1
SDIST = {"normal": 0, "unif": 1, "rademacher": 2}
PREC = {"fp32": 0, "bf16_sketch": 1, "fp8_sketch": 2}
ENGINE = {"auto": 0, "simt": 1, "tc": 2, "tc_tf32": 3}
LAYOUT = {"row": 0, "col": 1}

# Entry points declared in include/rsvdgb.h (checked by the ABI test).
EXPORTS = ["rsvdgb_create", "rsvdgb_destroy", "rsvdgb_set_stream", "rsvdgb_default_opts", "rsvdgb_status_string",
           "rsvdgb_sketch_width", "rsvdgb_rsvd", "rsvdgb_rsvd_host", "rsvdgb_rqb", "rsvdgb_omega",
           "rsvdgb_pass_ax", "rsvdgb_pass_atx", "rsvdgb_profile_passes", "rsvdgb_profile_read",
           "rsvdgb_kernel_launches", "rsvdgb_pass_atx_noalloc", "rsvdgb_test_pqr_barrier", "rsvdgb_rsvd_batched",
           "rsvdgb_default_train_opts", "rsvdgb_controller_load", "rsvdgb_controller_set",
           "rsvdgb_controller_train", "rsvdgb_controller_features", "rsvdgb_mlp_forward", "rsvdgb_mlp_grad",
           "rsvdgb_rpca", "rsvdgb_rpca_host", "rsvdgb_rid", "rsvdgb_rcur", "rsvdgb_default_rrpca_opts",
           "rsvdgb_rrpca"]

Q_MODE = {"fixed": 0, "learned": 1}
MLP_PARAMS = 5410  # RSVDGB_MLP_PARAMS
MLP_FEATURES = 16  # RSVDGB_MLP_FEATURES
MLP_TRAINABLE = MLP_PARAMS - 2 * MLP_FEATURES

# Static scratch of rsvdgb_pass_atx_noalloc (RSVDGB_NOALLOC_SCRATCH_BYTES).
NOALLOC_SCRATCH_BYTES = 16 << 20


class RsvdgbOpts(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("q", ctypes.c_int32), ("sdist", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("layout", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("q_mode", ctypes.c_int32), ("p_max", ctypes.c_int32), ("q_max", ctypes.c_int32),
                ("batched_eager", ctypes.c_int32), ("power", ctypes.c_int32), ("check_orth", ctypes.c_int32)]


class RsvdgbRrpcaOpts(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_float), ("tol", ctypes.c_float), ("rho", ctypes.c_float),
                ("maxiter", ctypes.c_int32), ("k0", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class RsvdgbRrpcaResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rank", ctypes.c_int32), ("k_next", ctypes.c_int32),
                ("status", ctypes.c_int32), ("err", ctypes.c_double), ("mu", ctypes.c_double),
                ("reserved", ctypes.c_double * 2)]


class RsvdgbTrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("tau", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 4)]


class RsvdgbInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("q_used", ctypes.c_int32), ("p_used", ctypes.c_int32),
                ("l", ctypes.c_int32), ("fro2_A", ctypes.c_double), ("fro2_B", ctypes.c_double),
                ("err2_QB", ctypes.c_double), ("err2_k", ctypes.c_double), ("breakdowns", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("jacobi_sweeps", ctypes.c_int32), ("orth_max", ctypes.c_float),
                ("reserved", ctypes.c_int32 * 4)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


INFO_BYTES = ctypes.sizeof(RsvdgbInfo)


class RsvdgbMatrixDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RsvdgbResultDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_void_p), ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64), ("V", ctypes.c_void_p),
                ("ldv", ctypes.c_int64)]

_lib = None


class RsvdgbError(RuntimeError):
    def __init__(self, where, status):
        super().__init__(f"{where} failed: {STATUS.get(status, status)}")
        self.status = status


def load(path: Path | str | None = None):
    """Load librsvdgb.so (build it first with paper_1608_02148_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build the CUDA library first (paper_1608_02148_gb300.build.build())")
    lib = ctypes.CDLL(str(p))
    P, I, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    lib.rsvdgb_create.argtypes = [ctypes.POINTER(P), I, P]
    lib.rsvdgb_destroy.argtypes = [P]
    lib.rsvdgb_set_stream.argtypes = [P, P]
    lib.rsvdgb_default_opts.argtypes = [ctypes.POINTER(RsvdgbOpts)]
    lib.rsvdgb_default_opts.restype = None
    lib.rsvdgb_status_string.argtypes = [I]
    lib.rsvdgb_status_string.restype = ctypes.c_char_p
    lib.rsvdgb_sketch_width.argtypes = [I64, I64, I, I]
    sig = [P, P, I64, I64, I64, I, I, I, I, ctypes.POINTER(RsvdgbOpts), P, P, I64, P, I64, P]
    lib.rsvdgb_rsvd.argtypes = sig
    lib.rsvdgb_rsvd_host.argtypes = sig
    pca_sig = [P, P, I64, I64, I64, I, I, I, I, ctypes.POINTER(RsvdgbOpts), P, I64, P, P, P, I64, P, P, P]
    lib.rsvdgb_rpca.argtypes = pca_sig
    lib.rsvdgb_rpca_host.argtypes = pca_sig
    lib.rsvdgb_default_rrpca_opts.argtypes = [ctypes.POINTER(RsvdgbRrpcaOpts)]
    lib.rsvdgb_default_rrpca_opts.restype = None
    lib.rsvdgb_rrpca.argtypes = [P, P, I64, I64, I64, ctypes.POINTER(RsvdgbRrpcaOpts), ctypes.POINTER(RsvdgbOpts), P,
                                 I64, P, I64, ctypes.POINTER(RsvdgbRrpcaResult)]
    lib.rsvdgb_rid.argtypes = [P, P, I64, I64, I64, I, I, ctypes.POINTER(RsvdgbOpts), P, I64, P, I64, P, P]
    lib.rsvdgb_rcur.argtypes = [P, P, I64, I64, I64, I, I, ctypes.POINTER(RsvdgbOpts), P, I64, P, I64, P, I64, P, P,
                                P]
    lib.rsvdgb_rqb.argtypes = [P, P, I64, I64, I64, I, I, ctypes.POINTER(RsvdgbOpts), P, I64, P, I64, P]
    lib.rsvdgb_omega.argtypes = [P, I64, I, U64, I, P, I64]
    lib.rsvdgb_pass_ax.argtypes = [P, P, I64, I64, I64, I, P, I64, I, P, I64, I, I]
    lib.rsvdgb_pass_atx.argtypes = [P, P, I64, I64, I64, I, P, I64, I, P, I64, I, I]
    lib.rsvdgb_profile_passes.argtypes = [P, I]
    lib.rsvdgb_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64),
                                        ctypes.POINTER(ctypes.c_double)]
    lib.rsvdgb_pass_atx_noalloc.argtypes = [P, P, I64, I64, I64, I, P, I64, I, P, I64]
    lib.rsvdgb_test_pqr_barrier.argtypes = [P, I64]
    lib.rsvdgb_rsvd_batched.argtypes = [P, I, ctypes.POINTER(RsvdgbMatrixDesc), I, ctypes.POINTER(RsvdgbOpts),
                                        ctypes.POINTER(RsvdgbResultDesc), P]
    lib.rsvdgb_kernel_launches.argtypes = []
    lib.rsvdgb_kernel_launches.restype = I64
    lib.rsvdgb_default_train_opts.argtypes = [ctypes.POINTER(RsvdgbTrainOpts)]
    lib.rsvdgb_default_train_opts.restype = None
    lib.rsvdgb_controller_load.argtypes = [P, ctypes.c_char_p]
    lib.rsvdgb_controller_set.argtypes = [P, P]
    lib.rsvdgb_controller_train.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(RsvdgbTrainOpts), ctypes.c_char_p,
                                            ctypes.POINTER(ctypes.c_float)]
    lib.rsvdgb_controller_features.argtypes = [P, P, I64, I64, I64, I, I, ctypes.POINTER(RsvdgbOpts), P]
    lib.rsvdgb_mlp_forward.argtypes = [P, P, P, I, P]
    lib.rsvdgb_mlp_grad.argtypes = [P, P, P, P, I, ctypes.c_float, P, P]
    _lib = lib
    return lib


def _check(where, rc):
    if rc != RSVDGB_OK:
        raise RsvdgbError(where, rc)


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _rowmajor_ld(t):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit column stride (row-major)")
    return t.stride(0)


POWER = {"subspace": 0, "lu": 1}


def make_opts(p=10, q=2, sdist="normal", prec="fp32", seed=0, layout="row", engine="auto", q_mode="fixed",
              p_max=None, q_max=None, power="subspace", check_orth=False) -> RsvdgbOpts:
    o = RsvdgbOpts()
    load().rsvdgb_default_opts(ctypes.byref(o))
    o.p, o.q, o.sdist, o.prec = p, q, SDIST[sdist], PREC[prec]
    o.power = POWER[power]
    o.seed, o.layout, o.engine = seed, LAYOUT[layout], ENGINE[engine]
    o.q_mode = Q_MODE[q_mode]
    o.check_orth = int(bool(check_orth))
    if p_max is not None:
        o.p_max = p_max
    if q_max is not None:
        o.q_max = q_max
    return o


def rsvdgb_default_opts() -> RsvdgbOpts:
    o = RsvdgbOpts()
    load().rsvdgb_default_opts(ctypes.byref(o))
    return o


def rsvdgb_status_string(status: int) -> str:
    return load().rsvdgb_status_string(status).decode()


def rsvdgb_sketch_width(m, n, k, p) -> int:
    return load().rsvdgb_sketch_width(m, n, k, p)


class Handle:
    """Owns an rsvdgb_handle bound to a device and (by default) torch's
    current stream on that device."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = ctypes.c_void_p()
        _check("rsvdgb_create", lib.rsvdgb_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)))
        self.ptr = h

    def close(self):
        if self.ptr:
            load().rsvdgb_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        _check("rsvdgb_set_stream", load().rsvdgb_set_stream(self.ptr, ctypes.c_void_p(stream.cuda_stream)))


def _info_from(buf) -> RsvdgbInfo:
    raw = bytes(buf.cpu().numpy().tobytes())
    return RsvdgbInfo.from_buffer_copy(raw)


def rsvdgb_rsvd(h: Handle, A, k, nu=-1, nv=-1, opts: RsvdgbOpts | None = None, out=None, sync_info=True):
    """rsvd(A, k, nu, nv, p, q, sdist) on a device tensor A (row-major unless
    opts.layout = col, where A is the column-major matrix given as its
    row-major transpose view).  Returns (d, U, V, info)."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    if opts.layout == LAYOUT["row"]:
        m, n = A.shape
        lda = _rowmajor_ld(A)
    else:  # column-major m x n matrix stored as the row-major n x m tensor A
        n, m = A.shape
        lda = _rowmajor_ld(A)
    nu_ = k if nu < 0 else nu
    nv_ = k if nv < 0 else nv
    dev = A.device
    if out is None:
        d = torch.empty(k, dtype=torch.float32, device=dev)
        U = torch.empty(m, max(nu_, 1), dtype=torch.float32, device=dev)
        V = torch.empty(n, max(nv_, 1), dtype=torch.float32, device=dev)
        info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=dev)
    else:
        d, U, V, info = out
    rc = lib.rsvdgb_rsvd(h.ptr, A.data_ptr(), m, n, lda, _dtype_code(A), k, nu_, nv_, ctypes.byref(opts),
                         d.data_ptr(), U.data_ptr() if nu_ > 0 else None, U.stride(0),
                         V.data_ptr() if nv_ > 0 else None, V.stride(0), info.data_ptr())
    _check("rsvdgb_rsvd", rc)
    if not sync_info:
        return d, U[:, :nu_], V[:, :nv_], info
    return d, U[:, :nu_], V[:, :nv_], _info_from(info)


def rsvdgb_rsvd_host(h: Handle, A_host, k, nu=-1, nv=-1, opts: RsvdgbOpts | None = None, out=None):
    """Host-buffer variant: A_host, and the outputs, are CPU tensors (pin
    them for full copy bandwidth).  Synchronous."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    m, n = A_host.shape if opts.layout == LAYOUT["row"] else A_host.shape[::-1]
    lda = _rowmajor_ld(A_host)
    nu_ = k if nu < 0 else nu
    nv_ = k if nv < 0 else nv
    if out is None:
        pin = A_host.is_pinned()
        d = torch.empty(k, dtype=torch.float32, pin_memory=pin)
        U = torch.empty(m, max(nu_, 1), dtype=torch.float32, pin_memory=pin)
        V = torch.empty(n, max(nv_, 1), dtype=torch.float32, pin_memory=pin)
    else:
        d, U, V = out
    info = RsvdgbInfo()
    rc = lib.rsvdgb_rsvd_host(h.ptr, A_host.data_ptr(), m, n, lda, _dtype_code(A_host), k, nu_, nv_,
                              ctypes.byref(opts), d.data_ptr(), U.data_ptr() if nu_ > 0 else None, U.stride(0),
                              V.data_ptr() if nv_ > 0 else None, V.stride(0), ctypes.byref(info))
    _check("rsvdgb_rsvd_host", rc)
    return d, U[:, :nu_], V[:, :nv_], info


def _pca_shape(A, opts):
    if opts.layout == LAYOUT["row"]:
        m, n = A.shape
    else:  # column-major m x n matrix given as the row-major n x m tensor
        n, m = A.shape
    return m, n, _rowmajor_ld(A)


def rsvdgb_rpca(h: Handle, A, k, center=True, scale=True, retx=True, opts: RsvdgbOpts | None = None,
                sync_info=True):
    """rpca(A, k, center, scale, retx, p, q) on a device tensor A
    (observations x variables).  Returns a dict with rotation (n x k),
    eigvals, sdev, x (m x k, or None without retx), center, scale, info."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    m, n, lda = _pca_shape(A, opts)
    dev = A.device
    f32 = dict(dtype=torch.float32, device=dev)
    rot = torch.empty(n, k, **f32)
    eig = torch.empty(k, **f32)
    sdev = torch.empty(k, **f32)
    x = torch.empty(m, k, **f32) if retx else None
    cen = torch.empty(n, **f32)
    sca = torch.empty(n, **f32)
    info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=dev)
    rc = lib.rsvdgb_rpca(h.ptr, A.data_ptr(), m, n, lda, _dtype_code(A), k, int(bool(center)), int(bool(scale)),
                         ctypes.byref(opts), rot.data_ptr(), k, eig.data_ptr(), sdev.data_ptr(),
                         x.data_ptr() if retx else None, k, cen.data_ptr(), sca.data_ptr(), info.data_ptr())
    _check("rsvdgb_rpca", rc)
    return {"rotation": rot, "eigvals": eig, "sdev": sdev, "x": x, "center": cen, "scale": sca,
            "info": _info_from(info) if sync_info else info}


def rsvdgb_rpca_host(h: Handle, A_host, k, center=True, scale=True, retx=True, opts: RsvdgbOpts | None = None):
    """Host-buffer variant of rsvdgb_rpca (CPU tensors in and out; pin A_host
    for full copy bandwidth).  Synchronous."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    m, n, lda = _pca_shape(A_host, opts)
    pin = dict(dtype=torch.float32, pin_memory=A_host.is_pinned())
    rot = torch.empty(n, k, **pin)
    eig = torch.empty(k, **pin)
    sdev = torch.empty(k, **pin)
    x = torch.empty(m, k, **pin) if retx else None
    cen = torch.empty(n, **pin)
    sca = torch.empty(n, **pin)
    info = RsvdgbInfo()
    rc = lib.rsvdgb_rpca_host(h.ptr, A_host.data_ptr(), m, n, lda, _dtype_code(A_host), k, int(bool(center)),
                              int(bool(scale)), ctypes.byref(opts), rot.data_ptr(), k, eig.data_ptr(),
                              sdev.data_ptr(), x.data_ptr() if retx else None, k, cen.data_ptr(), sca.data_ptr(),
                              ctypes.byref(info))
    _check("rsvdgb_rpca_host", rc)
    return {"rotation": rot, "eigvals": eig, "sdev": sdev, "x": x, "center": cen, "scale": sca, "info": info}


def rsvdgb_rid(h: Handle, A, k, opts: RsvdgbOpts | None = None, idx_only=False, sync_info=True):
    """rid(A, k, p, q): returns dict C (m x k), Z (k x n), J (k,), info."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    m, n, lda = _pca_shape(A, opts)
    f32 = dict(dtype=torch.float32, device=A.device)
    C = None if idx_only else torch.empty(m, k, **f32)
    Z = None if idx_only else torch.empty(k, n, **f32)
    J = torch.empty(k, dtype=torch.int64, device=A.device)
    info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=A.device)
    rc = lib.rsvdgb_rid(h.ptr, A.data_ptr(), m, n, lda, _dtype_code(A), k, ctypes.byref(opts),
                        C.data_ptr() if C is not None else None, k, Z.data_ptr() if Z is not None else None, n,
                        J.data_ptr(), info.data_ptr())
    _check("rsvdgb_rid", rc)
    return {"C": C, "Z": Z, "J": J, "info": _info_from(info) if sync_info else info}


def rsvdgb_rcur(h: Handle, A, k, opts: RsvdgbOpts | None = None, idx_only=False, sync_info=True):
    """rcur(A, k, p, q): returns dict C (m x k), U (k x k), R (k x n), J, I, info."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    m, n, lda = _pca_shape(A, opts)
    f32 = dict(dtype=torch.float32, device=A.device)
    C = None if idx_only else torch.empty(m, k, **f32)
    U = None if idx_only else torch.empty(k, k, **f32)
    R = None if idx_only else torch.empty(k, n, **f32)
    J = torch.empty(k, dtype=torch.int64, device=A.device)
    I_ = torch.empty(k, dtype=torch.int64, device=A.device)
    info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=A.device)
    rc = lib.rsvdgb_rcur(h.ptr, A.data_ptr(), m, n, lda, _dtype_code(A), k, ctypes.byref(opts),
                         C.data_ptr() if C is not None else None, k, U.data_ptr() if U is not None else None, k,
                         R.data_ptr() if R is not None else None, n, J.data_ptr(), I_.data_ptr(), info.data_ptr())
    _check("rsvdgb_rcur", rc)
    return {"C": C, "U": U, "R": R, "J": J, "I": I_, "info": _info_from(info) if sync_info else info}


def make_rrpca_opts(lam=None, tol=1e-5, rho=1.5, maxiter=50, k0=2) -> RsvdgbRrpcaOpts:
    o = RsvdgbRrpcaOpts()
    load().rsvdgb_default_rrpca_opts(ctypes.byref(o))
    o.lam = 0.0 if lam is None else lam
    o.tol, o.rho, o.maxiter, o.k0 = tol, rho, maxiter, k0
    return o


def rsvdgb_rrpca(h: Handle, A, ropts: RsvdgbRrpcaOpts | None = None, opts: RsvdgbOpts | None = None, want_L=True):
    """rrpca(A, lambda, maxiter, tol, p, q) on a row-major FP32 device tensor:
    returns dict L (or None), S, result (iters, rank, err, mu, status)."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    ropts = ropts or make_rrpca_opts()
    m, n = A.shape
    S = torch.empty(m, n, dtype=torch.float32, device=A.device)
    L = torch.empty(m, n, dtype=torch.float32, device=A.device) if want_L else None
    res = RsvdgbRrpcaResult()
    rc = lib.rsvdgb_rrpca(h.ptr, A.data_ptr(), m, n, _rowmajor_ld(A), ctypes.byref(ropts), ctypes.byref(opts),
                          L.data_ptr() if L is not None else None, n, S.data_ptr(), n, ctypes.byref(res))
    _check("rsvdgb_rrpca", rc)
    return {"L": L, "S": S, "result": res}


def rsvdgb_rqb(h: Handle, A, k, opts: RsvdgbOpts | None = None):
    """Algorithm rqb: returns Q (m x l), B (l x n), info."""
    torch = _torch()
    lib = load()
    opts = opts or make_opts()
    m, n = A.shape
    l = rsvdgb_sketch_width(m, n, k, opts.p)
    Q = torch.empty(m, l, dtype=torch.float32, device=A.device)
    B = torch.empty(l, n, dtype=torch.float32, device=A.device)
    info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=A.device)
    rc = lib.rsvdgb_rqb(h.ptr, A.data_ptr(), m, n, _rowmajor_ld(A), _dtype_code(A), k, ctypes.byref(opts),
                        Q.data_ptr(), Q.stride(0), B.data_ptr(), B.stride(0), info.data_ptr())
    _check("rsvdgb_rqb", rc)
    return Q, B, _info_from(info)


def rsvdgb_omega(h: Handle, rows, l, seed=0, sdist="normal", device="cuda"):
    torch = _torch()
    out = torch.empty(rows, l, dtype=torch.float32, device=device)
    _check("rsvdgb_omega", load().rsvdgb_omega(h.ptr, rows, l, seed, SDIST[sdist], out.data_ptr(), out.stride(0)))
    return out


def _pass(fn, name, h, A, X, engine, prec, out_rows):
    torch = _torch()
    m, n = A.shape
    l = X.shape[1]
    Y = torch.empty(out_rows, l, dtype=torch.float32, device=A.device)
    rc = fn(h.ptr, A.data_ptr(), m, n, _rowmajor_ld(A), _dtype_code(A), X.data_ptr(), _rowmajor_ld(X), l,
            Y.data_ptr(), Y.stride(0), ENGINE[engine], PREC[prec])
    _check(name, rc)
    return Y


def rsvdgb_pass_ax(h: Handle, A, X, engine="auto", prec="fp32"):
    """Y = A X (X: n x l float32 row-major)."""
    return _pass(load().rsvdgb_pass_ax, "rsvdgb_pass_ax", h, A, X, engine, prec, A.shape[0])


def rsvdgb_pass_atx(h: Handle, A, X, engine="auto", prec="fp32"):
    """Z = A^T X (X: m x l float32 row-major)."""
    return _pass(load().rsvdgb_pass_atx, "rsvdgb_pass_atx", h, A, X, engine, prec, A.shape[1])


def rsvdgb_profile_passes(h: Handle, enable: bool = True):
    _check("rsvdgb_profile_passes", load().rsvdgb_profile_passes(h.ptr, 1 if enable else 0))


def rsvdgb_profile_read(h: Handle):
    """(summed pass-kernel time in ms, launches, algorithmic bytes of A)."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    b = ctypes.c_double()
    _check("rsvdgb_profile_read", load().rsvdgb_profile_read(h.ptr, ctypes.byref(ms), ctypes.byref(n),
                                                             ctypes.byref(b)))
    return ms.value, n.value, b.value


def rsvdgb_test_pqr_barrier(h: Handle, spin_ticks: int):
    """Arm the failure-detection test hook: the next rid / rcur call's pivoted
    QR runs with one CTA absent from its first grid barrier and waits bounded
    by spin_ticks clock ticks, so it reports RSVDGB_ERR_TIMEOUT."""
    _check("rsvdgb_test_pqr_barrier", load().rsvdgb_test_pqr_barrier(h.ptr, int(spin_ticks)))


def rsvdgb_kernel_launches() -> int:
    return int(load().rsvdgb_kernel_launches())


def rsvdgb_pass_atx_noalloc(A, X, Z=None, stream=None):
    """Z = A^T X with no device allocation inside the library (static
    scratch).  A: m x n (float32 or bfloat16, row-major, on a CUDA device);
    X: m x l float32 row-major on the same device; Z (optional, allocated here
    when None): n x l float32 with unit column stride on that device.  Every
    argument is checked here, before anything is queued, and the call runs
    with A's device current (the library looks up its scratch on the current
    device)."""
    torch = _torch()
    if not isinstance(A, torch.Tensor) or A.dim() != 2 or A.device.type != "cuda":
        raise ValueError("A must be a 2-D tensor on a CUDA device")
    m, n = A.shape
    lda = _rowmajor_ld(A)
    dt = _dtype_code(A)
    if not isinstance(X, torch.Tensor) or X.dim() != 2 or X.dtype != torch.float32 or X.shape[0] != m:
        raise ValueError(f"X must be a float32 matrix with {m} rows")
    if X.device != A.device:
        raise ValueError("X must be on A's device")
    ldx = _rowmajor_ld(X)
    l = X.shape[1]
    if Z is None:
        Z = torch.empty(n, l, dtype=torch.float32, device=A.device)
    if not isinstance(Z, torch.Tensor) or Z.dim() != 2 or tuple(Z.shape) != (n, l) or Z.dtype != torch.float32:
        raise ValueError(f"Z must be a float32 tensor of shape ({n}, {l})")
    if Z.device != A.device:
        raise ValueError("Z must be on A's device")
    ldz = _rowmajor_ld(Z)
    if m < 1 or n < 1 or l < 1:
        raise ValueError("empty A^T X")
    if n * ldz * 4 > NOALLOC_SCRATCH_BYTES:
        raise ValueError(f"A^T X with n={n}, ldz={ldz} needs {n * ldz * 4} bytes of scratch; "
                         f"the static scratch holds {NOALLOC_SCRATCH_BYTES}")
    with torch.cuda.device(A.device):
        if stream is None:
            stream = torch.cuda.current_stream(A.device)
        rc = load().rsvdgb_pass_atx_noalloc(ctypes.c_void_p(stream.cuda_stream), A.data_ptr(), m, n, lda, dt,
                                            X.data_ptr(), ldx, l, Z.data_ptr(), ldz)
    _check("rsvdgb_pass_atx_noalloc", rc)
    return Z


class BatchedCall:
    """Descriptors and output buffers of one batch, reusable across calls (the
    library caches its plan and CUDA graph per batch layout)."""

    def __init__(self, mats, k, with_uv=True):
        torch = _torch()
        self.mats = mats
        self.k = k
        B = len(mats)
        self.descs = (RsvdgbMatrixDesc * B)()
        self.outs = (RsvdgbResultDesc * B)()
        self.d, self.U, self.V = [], [], []
        dev = mats[0].device
        for b, A in enumerate(mats):
            m, n = A.shape
            self.descs[b].A = A.data_ptr()
            self.descs[b].m, self.descs[b].n, self.descs[b].lda = m, n, _rowmajor_ld(A)
            self.descs[b].dtype = _dtype_code(A)
            d = torch.empty(k, dtype=torch.float32, device=dev)
            U = torch.empty(m, k, dtype=torch.float32, device=dev) if with_uv else None
            V = torch.empty(n, k, dtype=torch.float32, device=dev) if with_uv else None
            self.outs[b].d = d.data_ptr()
            self.outs[b].U = U.data_ptr() if U is not None else None
            self.outs[b].ldu = k
            self.outs[b].V = V.data_ptr() if V is not None else None
            self.outs[b].ldv = k
            self.d.append(d)
            self.U.append(U)
            self.V.append(V)
        self.infos = torch.zeros(B * INFO_BYTES, dtype=torch.uint8, device=dev)

    def info(self, b):
        raw = self.infos[b * INFO_BYTES:(b + 1) * INFO_BYTES]
        return _info_from(raw)


def rsvdgb_rsvd_batched(h: Handle, call: BatchedCall, opts: RsvdgbOpts | None = None):
    """Batched rSVD of call.mats (k, opts shared); results land in call.d/U/V."""
    opts = opts or make_opts()
    rc = load().rsvdgb_rsvd_batched(h.ptr, len(call.mats), call.descs, call.k, ctypes.byref(opts), call.outs,
                                    call.infos.data_ptr())
    _check("rsvdgb_rsvd_batched", rc)
    return call


# ---------------------------------------------------------------- learned (q, p) controller
def rsvdgb_default_train_opts() -> RsvdgbTrainOpts:
    o = RsvdgbTrainOpts()
    load().rsvdgb_default_train_opts(ctypes.byref(o))
    return o


def rsvdgb_controller_load(h: Handle, path):
    _check("rsvdgb_controller_load", load().rsvdgb_controller_load(h.ptr, str(path).encode()))


def rsvdgb_controller_set(h: Handle, params):
    """params: host float32 array of MLP_PARAMS values."""
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != MLP_PARAMS:
        raise ValueError(f"expected {MLP_PARAMS} parameters")
    _check("rsvdgb_controller_set", load().rsvdgb_controller_set(h.ptr, a.ctypes.data))


def rsvdgb_controller_train(h: Handle, dataset_path, out_path, opts: RsvdgbTrainOpts | None = None) -> float:
    o = opts if opts is not None else rsvdgb_default_train_opts()
    loss = ctypes.c_float(0.0)
    _check("rsvdgb_controller_train", load().rsvdgb_controller_train(h.ptr, str(dataset_path).encode(), ctypes.byref(o),
                                                                     str(out_path).encode(), ctypes.byref(loss)))
    return float(loss.value)


def rsvdgb_controller_features(h: Handle, A, k, opts: RsvdgbOpts | None = None, out=None):
    """16 features of A (device float32 tensor), as the learned mode computes them."""
    torch = _torch()
    o = opts if opts is not None else rsvdgb_default_opts()
    m, n = A.shape
    f = out if out is not None else torch.empty(MLP_FEATURES, dtype=torch.float32, device=A.device)
    _check("rsvdgb_controller_features", load().rsvdgb_controller_features(
        h.ptr, A.data_ptr(), m, n, _rowmajor_ld(A), _dtype_code(A), k, ctypes.byref(o), f.data_ptr()))
    return f


def rsvdgb_mlp_forward(h: Handle, P, X):
    torch = _torch()
    X = X.contiguous()
    out = torch.empty(X.shape[0], 2, dtype=torch.float32, device=X.device)
    _check("rsvdgb_mlp_forward", load().rsvdgb_mlp_forward(h.ptr, P.data_ptr(), X.data_ptr(), X.shape[0],
                                                           out.data_ptr()))
    return out


def rsvdgb_mlp_grad(h: Handle, P, X, Y, tau=0.9):
    """Gradient of the mean pinball loss w.r.t. the trainable parameters, and the loss."""
    torch = _torch()
    X = X.contiguous()
    Y = Y.contiguous()
    grad = torch.empty(MLP_TRAINABLE, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check("rsvdgb_mlp_grad", load().rsvdgb_mlp_grad(h.ptr, P.data_ptr(), X.data_ptr(), Y.data_ptr(), X.shape[0],
                                                     ctypes.c_float(tau), grad.data_ptr(), loss.data_ptr()))
    return grad, loss
