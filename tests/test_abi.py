"""The C ABI library loads and exports every entry point include/cheb.h declares.

Runs without a GPU: it only builds (nvcc cross-compiles for sm_103a), loads
libcheb.so and calls argument checks that fail before any CUDA work.
"""
import ctypes as C
import os
import re
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# exported by the checked build (libcheb_check.so) only
CHECK_ONLY = {"cheb_check_selftest"}


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"CHEB_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2307_04688_gb300 import build as B
    B.build()
    from paper_2307_04688_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("cheb_create", "cheb_destroy", "cheb_last_error", "cheb_fit", "cheb_eval_grid",
              "cheb_eval_grid_host", "cheb_eval_points", "game_solve", "cheb_device_status", "cheb_version"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        if name in CHECK_ONLY:
            assert not hasattr(lib, name), name
        else:
            assert hasattr(lib, name), name


def test_checked_build_exports_every_declared_symbol(lib):
    from paper_2307_04688_gb300 import _lib
    chk = C.CDLL(_lib.LIB_CHECK_PATH)
    for name in declared_functions():
        assert hasattr(chk, name), name
    chk.cheb_version.restype = C.c_char_p
    assert chk.cheb_version().decode().endswith("+check")
    assert not lib.cheb_version().decode().endswith("+check")
    # its argument checks are the default build's
    assert chk.cheb_check_selftest(None) == 1
    n = (C.c_int32 * 2)(3, 3)
    assert chk.cheb_fit(None, 2, n, None, None, None) == 1


RECORD_CALLS = textwrap.dedent("""
    import ctypes as C, sys
    L = C.CDLL(sys.argv[1])
    n = (C.c_int32 * 2)(3, 3)
    m = (C.c_int32 * 2)(4, 4)
    a = (C.c_double * 2)(-1.0, -1.0)
    b = (C.c_double * 2)(1.0, 1.0)
    assert L.cheb_fit(None, 2, n, None, None, None) == 1
    assert L.cheb_eval_grid(None, 2, n, None, a, b, m, None, None, 0, None) == 1
    assert L.cheb_eval_points(None, 2, n, None, a, b, 4, None, None, 0, None) == 1
    assert L.game_solve(None, 1, None, None, None, None) == 1
    assert L.surrogate_train(None, None, None, 0, None, 0, 0, 0, 0, C.c_float(0.0), 0, None, None) == 1
""")


def test_nvtx_ranges_around_entry_points(lib, tmp_path):
    """Each entry point opens an NVTX range named after itself and closes it on
    every return path (here: argument errors, no GPU needed). An injection
    library built from tests/nvtx_recorder.c records the ranges."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    rec = str(tmp_path / "libnvtx_recorder.so")
    subprocess.check_call([gcc, "-shared", "-fPIC", "-O1", "-I" + os.path.join(cuda, "include"),
                           os.path.join(ROOT, "tests", "nvtx_recorder.c"), "-o", rec])
    out = tmp_path / "ranges.txt"
    from paper_2307_04688_gb300 import _lib
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, NVTX_RECORD_FILE=str(out))
    subprocess.check_call([sys.executable, "-c", RECORD_CALLS, _lib.LIB_PATH], env=env, timeout=120)
    lines = out.read_text().splitlines()
    pushes = [ln[5:] for ln in lines if ln.startswith("push ")]
    assert pushes == ["cheb_fit", "cheb_eval_grid", "cheb_eval_points", "game_solve", "surrogate_train"], lines
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        assert depth in (0, 1), lines
    assert depth == 0, lines


def test_argument_errors_without_gpu(lib):
    assert lib.cheb_version().decode().count(".") == 2
    n = (C.c_int32 * 2)(3, 3)
    assert lib.cheb_fit(None, 2, n, None, None, None) == 1          # CHEB_EINVAL: null context
    assert b"context" in lib.cheb_last_error()
    h = C.c_void_p()
    assert lib.cheb_create(None, 0) == 1
    # the host-buffer evaluation checks its context before touching any buffer
    m = (C.c_int32 * 2)(4, 4)
    a = (C.c_double * 2)(-1.0, -1.0)
    b = (C.c_double * 2)(1.0, 1.0)
    assert lib.cheb_eval_grid_host(None, 2, n, None, a, b, m, None, None, 0, None) == 1
    assert b"context" in lib.cheb_last_error()
