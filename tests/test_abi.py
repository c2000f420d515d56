"""The C-ABI library builds, loads and exports every symbol include/pt.h declares;
host-side argument validation rejects bad scalars before any CUDA work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(pt_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_01506_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_entry_points():
    names = declared_functions()
    for must in ("pt_prepare", "pt_maxnull_naive", "pt_sync", "pt_destroy", "pt_last_error"):
        assert must in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_prepare_rejects_bad_sizes_without_cuda(lib):
    lib.pt_prepare.restype = ctypes.c_int
    lib.pt_prepare.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.pt_last_error.restype = ctypes.c_char_p
    lib.pt_last_error.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    for n, ngrid, n1 in [(2, 10, 1), (10, 10, 0), (10, 10, 10), (2000, 10, 5), (10, 0, 5)]:
        st = lib.pt_prepare(fake, n, ngrid, None, n1, None, ctypes.byref(out))
        assert st == 1, (n, ngrid, n1)
        assert lib.pt_last_error(None)
    assert lib.pt_prepare(None, 10, 10, None, 5, None, ctypes.byref(out)) == 1


def test_null_context_rejected(lib):
    lib.pt_maxnull_naive.restype = ctypes.c_int
    lib.pt_maxnull_naive.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int64] + [ctypes.c_void_p] * 3
    assert lib.pt_maxnull_naive(None, None, 10, None, None, None) == 1
    lib.pt_sync.restype = ctypes.c_int
    lib.pt_sync.argtypes = [ctypes.c_void_p]
    assert lib.pt_sync(None) == 1
    lib.pt_num_voxels.restype = ctypes.c_int64
    lib.pt_num_voxels.argtypes = [ctypes.c_void_p]
    assert lib.pt_num_voxels(None) == -1
    lib.pt_destroy.argtypes = [ctypes.c_void_p]
    lib.pt_destroy(None)


def test_oracle_and_product_share_no_code():
    """The oracle never imports the product's CUDA binding, and the product never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1703_01506_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "oracle/" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "binding" not in txt and "libpt" not in txt, f


def test_noalloc_binding_rejects_wrong_shapes_before_any_call():
    """The allocation-free wrapper checks perms against X and the output sizes
    against P and v before it loads or calls the library (CPU tensors suffice:
    the checks come first)."""
    import torch
    from paper_1703_01506_gb300 import binding as B
    n, v, P = 12, 50, 8
    X = torch.zeros((n, v), dtype=torch.float32)
    perms = torch.zeros((P, n), dtype=torch.int32)
    mx = torch.zeros(P, dtype=torch.float32)
    am = torch.zeros(P, dtype=torch.int32)
    ct = torch.zeros(v, dtype=torch.int32)
    bad = [
        dict(perms=torch.zeros((P, n + 1), dtype=torch.int32)),   # row length != n
        dict(perms=torch.zeros(P * n, dtype=torch.int32)),        # not 2-D
        dict(perms=torch.zeros((P, n), dtype=torch.int64)),       # wrong dtype
        dict(maxnull=torch.zeros(P - 1, dtype=torch.float32)),    # too short
        dict(argmax=torch.zeros(P - 1, dtype=torch.int32)),
        dict(argmax=torch.zeros(P, dtype=torch.int64)),
        dict(counts=torch.zeros(v - 1, dtype=torch.int32)),
        dict(X=torch.zeros((n, v), dtype=torch.float64)),
    ]
    for kw in bad:
        args = dict(X=X, n1=6, perms=perms, maxnull=mx, argmax=am, counts=ct)
        args.update(kw)
        with pytest.raises(ValueError):
            B.pt_maxnull_naive_noalloc(**args)
