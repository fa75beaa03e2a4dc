"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/rsvdgb.h declares.  Only host-only calls are made here."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsvdgb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsvdgb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1608_02148_gb300 import build, rsvdgb
    build.build()
    return rsvdgb.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_the_declared_entry_points(lib):
    from paper_1608_02148_gb300 import rsvdgb
    assert sorted(rsvdgb.EXPORTS) == sorted(set(rsvdgb.EXPORTS))
    assert set(rsvdgb.EXPORTS) <= set(declared_functions())
    assert set(declared_functions()) <= set(rsvdgb.EXPORTS)


def test_struct_sizes_match_header(lib):
    from paper_1608_02148_gb300 import rsvdgb
    assert ctypes.sizeof(rsvdgb.RsvdgbOpts) == 56
    assert ctypes.sizeof(rsvdgb.RsvdgbInfo) == 80


def test_default_opts_are_the_papers(lib):
    """p = 10, q = 2, sdist = normal (Sec. 3.6 signature; Sec. 3.3 remark)."""
    from paper_1608_02148_gb300 import rsvdgb
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))["rsvd_defaults"]
    o = rsvdgb.rsvdgb_default_opts()
    assert o.p == gold["p"] and o.q == gold["q"]
    assert o.sdist == rsvdgb.SDIST[gold["sdist"]]
    assert o.prec == 0 and o.layout == 0 and o.seed == 0


def test_status_strings_and_sketch_width(lib):
    from paper_1608_02148_gb300 import rsvdgb
    assert rsvdgb.rsvdgb_status_string(0) == "RSVDGB_OK"
    assert rsvdgb.rsvdgb_status_string(4) == "RSVDGB_ERR_BREAKDOWN"
    assert rsvdgb.rsvdgb_status_string(99) == "RSVDGB_UNKNOWN_STATUS"
    assert rsvdgb.rsvdgb_sketch_width(2000, 1000, 20, 10) == 30
    assert rsvdgb.rsvdgb_sketch_width(100, 40, 35, 10) == 40


def test_null_handle_is_rejected_without_gpu(lib):
    assert lib.rsvdgb_destroy(None) == 1
    assert lib.rsvdgb_rsvd(None, None, 10, 10, 10, 0, 2, 2, 2, None, None, None, 0, None, 0, None) == 1


def test_rrpca_structs_and_defaults(lib):
    """rrpca(A, lambda = NULL, maxiter = 50, tol = 1e-5, p = 10, q = 2) of
    Sec. 5.4; k = 2 at the start (Algorithm rrpca step 1)."""
    from paper_1608_02148_gb300 import rsvdgb
    assert ctypes.sizeof(rsvdgb.RsvdgbRrpcaOpts) == 32
    assert ctypes.sizeof(rsvdgb.RsvdgbRrpcaResult) == 48
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))["rrpca_defaults"]
    o = rsvdgb.RsvdgbRrpcaOpts()
    lib.rsvdgb_default_rrpca_opts(ctypes.byref(o))
    assert o.maxiter == gold["maxiter"] and abs(o.tol - gold["tol"]) < 1e-12
    assert o.k0 == gold["k0"] and o.lam == 0.0  # 0: lambda = max(m, n)^(-1/2)


def test_new_entry_points_reject_a_null_handle(lib):
    assert lib.rsvdgb_rpca(None, None, 10, 10, 10, 0, 2, 1, 1, None, None, 2, None, None, None, 2, None, None,
                           None) == 1
    assert lib.rsvdgb_rid(None, None, 10, 10, 10, 0, 2, None, None, 2, None, 10, None, None) == 1
    assert lib.rsvdgb_rrpca(None, None, 10, 10, 10, None, None, None, 10, None, 10, None) == 1


def test_header_compiles_as_c():
    """include/rsvdgb.h is a plain C header (no C++ or CUDA types)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    res = subprocess.run([cc, "-std=c11", "-fsyntax-only", "-x", "c", HEADER], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


# Library plumbing with no operation of the method behind it.
_PLUMBING = {"rsvdgb_create", "rsvdgb_destroy", "rsvdgb_set_stream", "rsvdgb_status_string"}


def test_every_entry_point_cites_its_passage():
    """Each declared call's comment (the nearest one above it) cites the
    passage of the paper that defines its operation, or states that it has
    no counterpart in the paper; only handle plumbing is exempt."""
    text = open(HEADER).read()
    for m in re.finditer(r"^(?:int|void|const char\*|int64_t)\s+(rsvdgb_[a-z0-9_]+)\s*\(", text, flags=re.M):
        name = m.group(1)
        if name in _PLUMBING:
            continue
        before = text[:m.start()]
        end = before.rfind("*/")
        comment = before[before.rfind("/*", 0, end):end]
        assert re.search(r"Sec\. \d|Algorithm \w|Eq\. \w|counterpart|not part of the paper", comment), name


def test_product_path_fails_loudly_without_library_or_gpu(lib, tmp_path, monkeypatch):
    """No fallback: a missing library is an error, and so is a handle on a
    machine without a usable GPU (the C call reports it; nothing runs on the
    CPU instead)."""
    import torch

    from paper_1608_02148_gb300 import rsvdgb
    monkeypatch.setattr(rsvdgb, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        rsvdgb.load(tmp_path / "librsvdgb.so")
    monkeypatch.undo()
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        rsvdgb.Handle(0)
    h = ctypes.c_void_p()
    assert lib.rsvdgb_create(ctypes.byref(h), 0, None) == 3  # RSVDGB_ERR_CUDA
    assert not h.value
