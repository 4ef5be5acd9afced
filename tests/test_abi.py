"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/teno7.h declares (no compute call is made here)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared():
    text = (ROOT / "include" / "teno7.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:t7_status|const char \*)\s*(t7_\w+)\s*\(", text, re.M)))


def test_header_declares_the_hot_path_calls():
    names = declared()
    for want in ("t7_teno7_reconstruct", "t7_euler_rhs", "t7_rk3_step", "t7_cfl_dt", "t7_run", "t7_create"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1808_00037_gb300 import build as cuda_build
    lib_path = cuda_build.build()
    lib = ctypes.CDLL(str(lib_path))
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_binds_every_declared_symbol():
    from paper_1808_00037_gb300 import binding
    lib = binding.load()
    for name in declared():
        fn = getattr(lib, name)
        assert fn.restype is not None, name


def test_binding_refuses_missing_library(tmp_path):
    from paper_1808_00037_gb300 import binding
    with pytest.raises(RuntimeError):
        binding.load(tmp_path / "nope.so")
