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
