"""The C-ABI library builds for sm_103a, loads, and exports every function include/tersoff.h declares
(no compute calls: these tests run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "tersoff.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tersoff_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11474_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = header_functions()
    for required in ("tersoff_build_neighbors", "tersoff_eval", "tersoff_fitness", "tersoff_param_grad"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1909_11474_gb300 import binding
    assert sorted(binding.EXPORTED) == header_functions()


def test_binding_loads_library_and_sets_signatures(lib):
    from paper_1909_11474_gb300 import binding
    L = binding.load()
    assert L.tersoff_eval.restype is ctypes.c_int
    # null context is rejected on the host before any CUDA call
    assert L.tersoff_eval(None, None, 1, 32, None, None, None, None) == binding.E_ARG
    assert L.tersoff_last_error(None) == b""
