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


def test_profile_kinds_match_the_header():
    """The binding's list of profiling kinds sizes the arrays that
    ebit_profile_read fills: it must have EBIT_PROF_KINDS entries."""
    import os

    from paper_2509_26361_gb300 import ebit

    src = open(os.path.join(ROOT, "include", "ebit.h")).read()
    m = re.search(r"EBIT_PROF_KINDS\s*=\s*(\d+)", src)
    assert m and int(m.group(1)) == len(ebit.PROF_KINDS)
