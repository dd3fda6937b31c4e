"""The C-ABI library builds, loads and exports exactly what include/lp.h
declares; argument checks that need no device (CPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2301_09125_gb300 import build

    build.build()
    import paper_2301_09125_gb300 as lp

    return lp.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["lp_graph_create", "lp_rak_run", "lp_modularity", "lp_labels_get",
                     "lp_batch_create", "lp_batch_run", "lp_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2301_09125_gb300 as lp

    out = subprocess.run(["nm", "-D", "--defined-only", lp._binding.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (lp_[a-z_]+)$", out, flags=re.M))
    declared = set(declared_functions())
    assert declared <= exported, declared - exported
    assert declared == set(lp.SIGNATURES), set(lp.SIGNATURES) ^ declared
    for name in declared:
        assert getattr(lib, name) is not None


def test_header_compiles_as_c():
    src = '#include "lp.h"\nint main(void){lp_rak_params p; return lp_rak_params_default(&p);}\n'
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-x", "c", "-", "-fsyntax-only"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_params_default_and_argument_checks(lib):
    import paper_2301_09125_gb300 as lp

    p = lp.lp_rak_params_default()
    assert p.tolerance == 0.05 and p.max_iter == 20 and p.mode == lp.LP_SYNC and p.strict == 1
    assert lib.lp_rak_params_default(None) == lp.LP_EINVAL
    assert "NULL" in lp.lp_last_error()
    h = ctypes.c_void_p()
    off = (ctypes.c_int32 * 2)(0, 0)
    assert lib.lp_graph_create(-1, 0, off, None, None, 0, None, ctypes.byref(h)) == lp.LP_EINVAL
    assert "n must be" in lp.lp_last_error()
    assert lib.lp_graph_create(1, -5, off, None, None, 0, None, ctypes.byref(h)) == lp.LP_EINVAL
    assert lib.lp_graph_create(1, 0, None, None, None, 0, None, ctypes.byref(h)) == lp.LP_EINVAL
    assert lib.lp_graph_create(1, 0, off, None, None, lp.LP_FLAG_BORROW, None,
                               ctypes.byref(h)) == lp.LP_EINVAL
    assert lib.lp_graph_create(1, 0, off, None, None, 0x100, None, ctypes.byref(h)) == lp.LP_EINVAL
    assert h.value is None
    assert lib.lp_graph_destroy(None) == lp.LP_OK
    assert lib.lp_batch_destroy(None) == lp.LP_OK
    assert lib.lp_rak_run(None, ctypes.byref(p), None) == lp.LP_EINVAL
    assert lib.lp_batch_create(0, None, 0, None, ctypes.byref(h)) == lp.LP_EINVAL
    assert lp.lp_launch_count() >= 0


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2301_09125_gb300._binding as b

    saved = b._lib
    b._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            b.load(str(tmp_path / "missing.so"))
    finally:
        b._lib = saved
