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
