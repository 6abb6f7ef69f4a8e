"""bst_grad_loglike_noalloc: the gradient call for programs that must not allocate
device memory while running (their memory belongs to a caching allocator or a
budget fixed at start-up).  It keeps the adjoint's activations in the library's
16 MiB static device array instead of allocating, and must return what
bst_grad_loglike returns.  This file is collected last on purpose, and passes
alone in a fresh process as well as after the other tests."""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu

# same tolerances as the loglike parity tests (relative to the reference output)
TOL = {"fp64": (1e-10, 1e-9), "fp32": (1e-5, 1e-4), "bf16": (2e-3, 2e-2)}


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp64"])
def test_noalloc_gradient_matches_grad_loglike_twice(prec):
    from paper_2606_04895_gb300 import Sampler, _lib
    d, width, depth = 8, 512, 4
    e = S.emulator(d, width=width, depth=depth, seed=5, out_m=50.0, out_s=10.0)
    s = Sampler(d, 16, precision=prec, likelihood="emulator", seed=3)
    s.set_emulator(e["params"], depth, width, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    tl, tg = TOL[prec]
    for call, m in enumerate((300, 1000)):
        x = torch.as_tensor(np.random.default_rng(call).uniform(-3, 3, (m, d)), dtype=s.dtype, device="cuda")
        ll_ref, g_ref = s.grad_loglike(x)
        ll = torch.full((m,), float("nan"), dtype=s.dtype, device="cuda")
        g = torch.full((m, d), float("nan"), dtype=s.dtype, device="cuda")
        rc = s.lib.bst_grad_loglike_noalloc(s.h, _ptr(x), m, _ptr(ll), _ptr(g), stream)
        assert rc == _lib.OK, s.lib.bst_last_error()
        torch.cuda.synchronize()
        err_l = ((ll - ll_ref).abs() / ll_ref.abs().clamp_min(1.0)).max().item()
        err_g = ((g - g_ref).abs().max() / g_ref.abs().max()).item()
        assert err_l <= tl and err_g <= tg, (call, err_l, err_g)
    # more points than the static array holds: refused before any launch
    big = 16 * 1024 * 1024 // ((depth - 1) * width * (2 if prec == "bf16" else s.dtype.itemsize)) + 1
    rc = s.lib.bst_grad_loglike_noalloc(s.h, _ptr(x), big, _ptr(ll), _ptr(g), stream)
    assert rc == _lib.ERR_ARG and b"static scratch" in s.lib.bst_last_error()
    s.close()


def test_noalloc_bf16_without_room_for_exchange_images():
    """4800 points of a BF16 8-512x4-1 emulator run on clusters of four CTAs, whose exchange
    images no longer fit in the static array beside the activations: the call then uses the
    shared->shared exchange and must still return what bst_grad_loglike returns."""
    from paper_2606_04895_gb300 import Sampler, _lib
    d, width, depth, m = 8, 512, 4, 4800
    e = S.emulator(d, width=width, depth=depth, seed=6, out_m=50.0, out_s=10.0)
    s = Sampler(d, 16, precision="bf16", likelihood="emulator", seed=3)
    s.set_emulator(e["params"], depth, width, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.as_tensor(np.random.default_rng(7).uniform(-3, 3, (m, d)), dtype=s.dtype, device="cuda")
    ll_ref, g_ref = s.grad_loglike(x)
    ll = torch.full((m,), float("nan"), dtype=s.dtype, device="cuda")
    g = torch.full((m, d), float("nan"), dtype=s.dtype, device="cuda")
    rc = s.lib.bst_grad_loglike_noalloc(s.h, _ptr(x), m, _ptr(ll), _ptr(g), stream)
    assert rc == _lib.OK, s.lib.bst_last_error()
    torch.cuda.synchronize()
    tl, tg = TOL["bf16"]
    err_l = ((ll - ll_ref).abs() / ll_ref.abs().clamp_min(1.0)).max().item()
    err_g = ((g - g_ref).abs().max() / g_ref.abs().max()).item()
    assert err_l <= tl and err_g <= tg, (err_l, err_g)
    s.close()
