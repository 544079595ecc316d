"""The C-ABI library builds, loads and exports every symbol that the
public headers declare (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2410_03969_gb300 as rp
from paper_2410_03969_gb300 import build as rpbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rpchol_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    rpbuild.build()
    return ctypes.CDLL(rpbuild.LIB)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for required in ("rpchol_create", "rpchol_run", "rpchol_factor", "rpchol_run_plain",
                     "rpchol_copy_factor", "rpchol_stats", "rpchol_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in declared_symbols() if not hasattr(library, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_core(library):
    bound = {n for n, _, _ in rp._SIGNATURES}
    for n in ("rpchol_create", "rpchol_run", "rpchol_run_plain", "rpchol_factor",
              "rpchol_copy_factor", "rpchol_stats", "rpchol_destroy"):
        assert n in bound


def test_version_string_without_gpu(library):
    library.rpchol_version.restype = ctypes.c_char_p
    assert b"sm_103a" in library.rpchol_version()


def test_invalid_arguments_are_rejected_before_any_launch(library):
    rp.lib()
    ctx = ctypes.c_void_p()
    x = (ctypes.c_float * 8)()
    # sigma <= 0, k_max > N, T_max > 256, d < 1: EINVAL with no device work
    for args in ((0, -1.0, 4, 2, 2, 4), (0, 1.0, 4, 2, 5, 4), (0, 1.0, 4, 2, 2, 300),
                 (0, 1.0, 4, 0, 2, 4), (7, 1.0, 4, 2, 2, 4)):
        kind, sigma, N, d, kmax, tmax = args
        rc = rp.lib().rpchol_create(kind, sigma, ctypes.cast(x, ctypes.c_void_p), N, d, 0, 0,
                                    kmax, tmax, None, ctypes.byref(ctx))
        assert rc == 1, args
        assert rp.lib().rpchol_last_error()
    assert rp.lib().rpchol_run(None, 1, 1, 0) == 1


def test_binding_binds_every_declared_symbol():
    bound = {n for n, _, _ in rp._SIGNATURES}
    missing = [n for n in declared_symbols() if n not in bound]
    assert not missing, missing


def test_invalid_arguments_of_the_other_algorithms(library):
    L = rp.lib()
    out = ctypes.c_void_p()
    x = (ctypes.c_float * 64)()
    xp = ctypes.cast(x, ctypes.c_void_p)
    # block RPCholesky on no context
    assert L.rpchol_run_block(None, 1, 1, 0) == 1
    # low memory: k_max > N, k_max > 16384, T_max > 256, bad kind, bad dtype
    for kind, sigma, N, d, dt, kmax, tmax in ((0, 1.0, 8, 2, 0, 9, 4),
                                             (0, 1.0, 20000, 2, 0, 16385, 4),
                                             (0, 1.0, 8, 2, 0, 4, 257),
                                             (5, 1.0, 8, 2, 0, 4, 4),
                                             (0, 1.0, 8, 2, 3, 4, 4)):
        assert L.rpchol_lowmem_create(kind, sigma, xp, N, d, dt, kmax, tmax, None,
                                      ctypes.byref(out)) == 1
        assert not out.value
    assert L.rpchol_lowmem_run(None, 1, 1, 0) == 1
    assert L.rpchol_lowmem_copy(None, None, 0, None, None, None, None) == 1
    assert L.rpchol_lowmem_destroy(None) == 0
    # RPQR: ldb < M, k_max > min(M, N), T_max > 256
    b = (ctypes.c_double * 64)()
    bp = ctypes.cast(b, ctypes.c_void_p)
    for M, N, ldb, kmax, tmax in ((8, 8, 4, 2, 2), (4, 16, 4, 5, 2), (8, 8, 8, 2, 257)):
        assert L.rpchol_rpqr_create(bp, M, N, ldb, kmax, tmax, None, ctypes.byref(out)) == 1
    assert L.rpchol_rpqr_run(None, 1, 1, 0) == 1
    assert L.rpchol_rpqr_copy(None, None, 0, None, 0, None, None, None, None) == 1
    assert L.rpchol_rpqr_destroy(None) == 0


def test_checkpoint_calls_reject_bad_arguments(library):
    L = rp.lib()
    n = ctypes.c_size_t(0)
    assert L.rpchol_save(None, None, ctypes.byref(n)) == 1
    buf = ctypes.create_string_buffer(16)
    assert L.rpchol_restore(None, buf, 16) == 1
    assert L.rpchol_resume(None, 10) == 1


def test_selftest_limit_is_checked_before_any_launch(library):
    assert rp.lib().rpchol_selftest_wait(0, None) == 1
    assert rp.lib().rpchol_selftest_wait(2001, None) == 1


def test_header_is_plain_c(tmp_path):
    """include/rpchol.h compiles as C11 (no C++ or torch types cross the
    boundary) and a C program linking every declared entry point links."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    names = declared_symbols()
    src = tmp_path / "use.c"
    body = "\n".join("    (void *)&%s," % n for n in names)
    src.write_text('#include "rpchol.h"\n#include <stddef.h>\n'
                   "void *table[] = {\n%s\n    NULL};\nint main(void) { return table[0] == NULL; }\n"
                   % body)
    rpbuild.build()
    out = tmp_path / "use"
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(out), rpbuild.LIB,
                        "-Wl,-rpath," + os.path.dirname(rpbuild.LIB)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
