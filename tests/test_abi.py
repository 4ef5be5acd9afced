"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point the headers under include/ declare (no compute call is made here)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared():
    names = set()
    for h in sorted((ROOT / "include").glob("*.h")):
        text = h.read_text()
        names |= set(re.findall(r"^\s*(?:t7_status|const char \*)\s*(t7_\w+)\s*\(", text, re.M))
    return sorted(names)


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


def test_checked_build_builds_and_exports_every_declared_symbol():
    """The index-checked build (T7_CHECKED=1) compiles from the same sources
    and offers the same entry points (its GPU runs: test_gpu_checked.py)."""
    from paper_1808_00037_gb300 import build as cuda_build
    lib_path = cuda_build.build(checked=True)
    assert lib_path.name == "libteno7_checked.so"
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


def test_grid_struct_layout_matches_header(tmp_path):
    """The binding's t7_grid has the C struct's size and field offsets (a C
    program compiled against the header prints them)."""
    import shutil
    import subprocess
    from paper_1808_00037_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in binding.t7_grid._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"teno7.h\"\nint main(void){\n"
                   "printf(\"%zu\\n\", sizeof(t7_grid));\n"
                   + "".join(f"printf(\"%zu\\n\", offsetof(t7_grid, {f}));\n" for f in fields) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(binding.t7_grid)
    assert out[1:] == [getattr(binding.t7_grid, f).offset for f in fields]


def test_create_rejects_bad_scheme_without_touching_the_device():
    """t7_create validates the grid before any CUDA call: an unknown scheme, and
    the TENO5 baseline on the 2D system, are refused with T7_EINVAL."""
    from paper_1808_00037_gb300 import binding as B
    lib = B.load()
    bc = (ctypes.c_int * 4)(0, 0, 0, 0)
    h = ctypes.c_void_p()
    g = B.t7_grid(B.T7_EULER1D, B.T7_F64, 64, 1, 0.1, 0.0, bc, 1.4, 1.0, 1e-5, -1.0, -1.0, 7)
    assert lib.t7_create(ctypes.byref(g), None, ctypes.byref(h)) == B.T7_EINVAL
    g = B.t7_grid(B.T7_EULER2D, B.T7_F64, 64, 64, 0.1, 0.1, bc, 1.4, 1.0, 1e-5, -1.0, -1.0, B.T7_TENO5)
    assert lib.t7_create(ctypes.byref(g), None, ctypes.byref(h)) == B.T7_EINVAL
    assert not h.value


def test_create_rejects_empty_and_oversized_grids_without_touching_the_device():
    """nx or ny < 1, a 1D grid with ny != 1, and grids whose m * nx * ny exceeds
    the 32-bit index range the kernels use are refused with T7_EINVAL before
    any allocation."""
    from paper_1808_00037_gb300 import binding as B
    lib = B.load()
    bc = (ctypes.c_int * 4)(0, 0, 0, 0)
    h = ctypes.c_void_p()
    for sys_, nx, ny in ((B.T7_EULER1D, 0, 1), (B.T7_EULER1D, 16, 2), (B.T7_EULER2D, 16, 0),
                         (B.T7_EULER1D, 715_827_883, 1), (B.T7_EULER2D, 23_171, 23_171)):
        g = B.t7_grid(sys_, B.T7_F32, nx, ny, 0.1, 0.1, bc, 1.4, 1.0, 1e-5, -1.0, -1.0)
        assert lib.t7_create(ctypes.byref(g), None, ctypes.byref(h)) == B.T7_EINVAL, (sys_, nx, ny)
        assert not h.value


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """include/teno7.h compiles as strict C99 (-Wall -Wextra -pedantic, no
    warnings), and a C program linked against libteno7 calls t7_create with an
    empty grid and gets T7_EINVAL back (no device work on that path)."""
    import shutil
    import subprocess
    from paper_1808_00037_gb300 import build as cuda_build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_path = cuda_build.build()
    src = tmp_path / "use.c"
    src.write_text('#include "teno7.h"\n#include "teno7_probe.h"\n'
                   "int main(void) {\n"
                   "    t7_grid g = {0};\n"
                   "    t7_ctx *c = 0;\n"
                   "    g.sys = T7_EULER1D; g.prec = T7_F32; g.nx = 0; g.ny = 1; g.dx = 1.0;\n"
                   "    return t7_create(&g, 0, &c) == T7_EINVAL && c == 0 ? 0 : 1;\n"
                   "}\n")
    exe = tmp_path / "use"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", str(ROOT / "include"),
                        str(src), "-L", str(lib_path.parent), "-lteno7", f"-Wl,-rpath,{lib_path.parent}",
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0
