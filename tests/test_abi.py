"""The C-ABI library builds, loads and exports every symbol include/bst.h declares;
host-side argument checks return their status codes without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bst_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["bst_create", "bst_init_chains", "bst_step", "bst_loglike", "bst_grad_loglike", "bst_adapt_cov"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2606_04895_gb300 import _lib
    L = _lib.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(_lib.SYMBOLS) == _declared()
    assert L.bst_version().decode().startswith("bst")


def test_host_side_argument_errors():
    from paper_2606_04895_gb300 import _lib
    L = _lib.load()
    h = C.c_void_p()
    assert L.bst_create(C.byref(h), None) == _lib.ERR_ARG
    cfg = _lib.Config(d=0, n_chains=8, precision=_lib.FP32, lik_kind=_lib.LIK_EMULATOR)
    assert L.bst_create(C.byref(h), C.byref(cfg)) == _lib.ERR_ARG
    assert b"d must be" in L.bst_last_error()
    cfg = _lib.Config(d=4, n_chains=8, precision=_lib.BF16, lik_kind=_lib.LIK_ANALYTIC)
    assert L.bst_create(C.byref(h), C.byref(cfg)) == _lib.ERR_UNSUPPORTED
    cfg = _lib.Config(d=4, n_chains=8, precision=_lib.FP32, lik_kind=_lib.LIK_EMULATOR, max_depth=11)
    assert L.bst_create(C.byref(h), C.byref(cfg)) == _lib.ERR_ARG
    assert L.bst_step(None, 0, 0.1, 1, 1, None, None, None) == _lib.ERR_ARG
    assert L.bst_sync(None, None) == _lib.ERR_ARG
    L.bst_destroy(None)


def test_ctypes_mirrors_match_the_header_layout(tmp_path):
    """The binding's ctypes structures and enum values against the C compiler's view of
    include/bst.h (sizes, field offsets, enum values), so the two cannot drift apart."""
    import shutil
    import subprocess
    from paper_2606_04895_gb300 import _lib
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    cfg_fields = [f for f, _ in _lib.Config._fields_]
    st_fields = [f for f, _ in _lib.StepStats._fields_]
    kernels = ["BST_MH", "BST_MALA", "BST_HMC", "BST_NUTS", "BST_AIES", "BST_AIES_DE", "BST_NUTS_MULTINOMIAL", "BST_BF16", "BST_FP32", "BST_FP64",
               "BST_FP16"]
    statuses = ["BST_OK", "BST_ERR_ARG", "BST_ERR_STATE", "BST_ERR_CUDA", "BST_ERR_NOT_PD", "BST_ERR_TIMEOUT",
                "BST_ERR_NONFINITE", "BST_ERR_UNSUPPORTED"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bst.h"', "int main(void) {",
             '  printf("cfg %zu\\n", sizeof(bst_config));', '  printf("st %zu\\n", sizeof(bst_step_stats));']
    lines += [f'  printf("cfg.{f} %zu\\n", offsetof(bst_config, {f}));' for f in cfg_fields]
    lines += [f'  printf("st.{f} %zu\\n", offsetof(bst_step_stats, {f}));' for f in st_fields]
    lines += [f'  printf("{k} %d\\n", (int){k});' for k in kernels + statuses]
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert int(got["cfg"]) == C.sizeof(_lib.Config)
    assert int(got["st"]) == C.sizeof(_lib.StepStats)
    for f in cfg_fields:
        assert int(got[f"cfg.{f}"]) == getattr(_lib.Config, f).offset, f
    for f in st_fields:
        assert int(got[f"st.{f}"]) == getattr(_lib.StepStats, f).offset, f
    for k in kernels:
        assert int(got[k]) == getattr(_lib, k[4:]), k
    for sname in statuses:
        assert int(got[sname]) == getattr(_lib, sname[4:]), sname


def test_every_entry_point_rejects_a_null_handle():
    """Each call that takes a handle returns BST_ERR_ARG for a NULL one, before any device
    work, and names itself in the error message."""
    from paper_2606_04895_gb300 import _lib
    L = _lib.load()
    skip = {"bst_version", "bst_last_error", "bst_create", "bst_destroy", "bst_r_minus_1_combine"}
    ints = (C.c_int, C.c_longlong, C.c_ulonglong, C.c_uint32, C.c_uint64)
    for name in _lib.SYMBOLS:
        if name in skip:
            continue
        f = getattr(L, name)
        args = [0 if t in ints else 0.0 if t is C.c_double else None for t in f.argtypes]
        assert f(*args) == _lib.ERR_ARG, name
        assert L.bst_last_error().decode().startswith(name + ":"), (name, L.bst_last_error())
    L.bst_destroy(None)  # a no-op
