"""The C-ABI library builds, loads and exports every entry point of include/cpm.h (CPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cpm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_solver_entry_points():
    names = _declared()
    for n in ["cpm_build_band", "cpm_build_hierarchy", "cpm_apply", "cpm_smooth", "cpm_vcycle",
              "cpm_solve", "cpm_residual", "cpm_solve_batch", "cpm_mlp_train", "cpm_mlp_save",
              "cpm_mlp_load"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1307_4354_gb300 as pkg
    path = pkg.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (cpm_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = pkg.capi.lib()
    for n in _declared():
        assert hasattr(lib, n)
    assert set(pkg.capi.exported_names()) == set(_declared())


def test_status_strings_without_gpu():
    import paper_1307_4354_gb300 as pkg
    pkg.build()
    assert pkg.capi.cpm_status_str(0) == "ok"
    assert "reach" in pkg.capi.cpm_status_str(4)


def test_no_oracle_in_product_path():
    """The package never imports the oracle (test infrastructure only)."""
    pkgdir = os.path.join(ROOT, "paper_1307_4354_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_null_handles_are_rejected_without_a_gpu():
    """Every entry point checks its handles before any device work: NULL gives
    CPM_ERR_ARG with a message, destroy(NULL) is a no-op (CPU only)."""
    import ctypes as C
    import paper_1307_4354_gb300 as pkg
    pkg.build()
    L = pkg.capi.lib()
    ERR_ARG = pkg.capi.CPM_ERR_ARG
    out = C.c_void_p()
    assert L.cpm_build_hierarchy(None, None, None, C.byref(out)) == ERR_ARG
    assert L.cpm_solve(None, None, None, None, None, None) == ERR_ARG
    assert L.cpm_residual_norms_noalloc(None, None, None, None, None) == ERR_ARG
    assert L.cpm_build_batch(None, 0, 1, None, C.byref(out)) == ERR_ARG
    assert L.cpm_build_batch(None, 1, 0, None, C.byref(out)) == ERR_ARG
    assert L.cpm_solve_batch(None, None, None, None, None, None) == ERR_ARG
    assert L.cpm_batch_info(None, None, None) == ERR_ARG
    assert L.cpm_last_error()
    assert L.cpm_batch_destroy(None) == pkg.capi.CPM_OK
