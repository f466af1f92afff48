"""The C ABI library builds for sm_103a, loads, and exports every function include/kitrt.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(kitrt_\w+)\s*\(", text)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2205_08417_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2205_08417_gb300 import kitrt
    names = declared_functions()
    assert set(names) == set(kitrt.SIGNATURES), set(names) ^ set(kitrt.SIGNATURES)


def test_host_only_entry_points():
    """Entry points that touch no device: status strings and default parameters."""
    from paper_2205_08417_gb300 import build, kitrt
    build.build()
    L = kitrt._lib()
    assert L.kitrt_status_string(0) == b"ok"
    assert L.kitrt_status_string(4).startswith(b"Hessian")
    p = kitrt.Params()
    assert L.kitrt_default_params(ctypes.byref(p)) == 0
    assert p.degree == 2 and p.quad_order == 10 and abs(p.tau - 1e-10) < 1e-25
    assert L.kitrt_default_params(None) == 1
    # null handles are rejected on the host before any CUDA call
    assert L.kitrt_mesh_create(None, 0, None, 0, None) == 1
    assert L.kitrt_mn_init(None, None, None) == 1
    assert L.kitrt_step(None, None, None, None, None, None, 0.0, 1, None, None, None) == 1
