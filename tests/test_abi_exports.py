"""The C ABI library builds for sm_103a and exports every function that
include/ebit.h declares (no GPU needed: symbols only, no compute calls)."""
import ctypes
import os
import re

from paper_2509_26361_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    out = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ebit_[a-z0-9_]+)\s*\(", src, re.M):
            out.add(m.group(1))
    return out


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"ebit_create", "ebit_advect_sweep", "ebit_front2vof", "ebit_curvature"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_gpu():
    import pytest
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_26361_gb300 import ebit

    with pytest.raises(Exception):
        ebit.Grid(16, 16, 16)
