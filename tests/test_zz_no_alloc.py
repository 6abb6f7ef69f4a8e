"""bst_grad_loglike_noalloc: the gradient call for programs that must not allocate
device memory while running (their memory belongs to a caching allocator or a
budget fixed at start-up).  It keeps the adjoint's activations in the library's
16 MiB static device array instead of allocating.  It runs the same kernels on
the same tiles as bst_grad_loglike, with only the place of the stored
activations changed, so its results must equal bst_grad_loglike's bit for bit.
This file is collected last on purpose, and passes alone in a fresh process as
well as after the other tests."""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _call(s, x, m):
    from paper_2606_04895_gb300 import _lib
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ll = torch.full((m,), float("nan"), dtype=s.dtype, device="cuda")
    g = torch.full((m, s.d), float("nan"), dtype=s.dtype, device="cuda")
    rc = s.lib.bst_grad_loglike_noalloc(s.h, _ptr(x), m, _ptr(ll), _ptr(g), stream)
    assert rc == _lib.OK, s.lib.bst_last_error()
    torch.cuda.synchronize()
    return ll, g


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp64"])
def test_noalloc_gradient_matches_grad_loglike_twice(prec):
    from paper_2606_04895_gb300 import Sampler, _lib
    d, width, depth = 8, 512, 4
    e = S.emulator(d, width=width, depth=depth, seed=5, out_m=50.0, out_s=10.0)
    s = Sampler(d, 16, precision=prec, likelihood="emulator", seed=3)
    s.set_emulator(e["params"], depth, width, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    # two calls in a row, the second larger: the array keeps the first call's contents
    for call, m in enumerate((300, 1000)):
        x = torch.as_tensor(np.random.default_rng(call).uniform(-3, 3, (m, d)), dtype=s.dtype, device="cuda")
        ll_ref, g_ref = s.grad_loglike(x)
        ll, g = _call(s, x, m)
        assert torch.equal(ll, ll_ref) and torch.equal(g, g_ref), call
    # more points than the static array holds: refused before any launch
    big = 16 * 1024 * 1024 // ((depth - 1) * width * (2 if prec == "bf16" else s.dtype.itemsize)) + 1
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = s.lib.bst_grad_loglike_noalloc(s.h, _ptr(x), big, _ptr(ll), _ptr(g), stream)
    assert rc == _lib.ERR_ARG and b"static scratch" in s.lib.bst_last_error()
    s.close()


@pytest.mark.parametrize("width,depth,m", [(512, 4, 5461), (512, 8, 2000)])
def test_noalloc_bf16_near_the_limit(width, depth, m):
    """The largest point count the array holds for a BF16 8-512x4-1 emulator (5461 points: 43
    tiles, clusters of two CTAs, whose stored activations go to the array), and an 8-deep
    width-512 emulator (too deep for the tensor memory of a 4-CTA cluster: clusters of two,
    activations in the array): both equal bst_grad_loglike bit for bit, twice in a row."""
    from paper_2606_04895_gb300 import Sampler
    d = 8
    e = S.emulator(d, width=width, depth=depth, seed=6, out_m=50.0, out_s=10.0)
    s = Sampler(d, 16, precision="bf16", likelihood="emulator", seed=3)
    s.set_emulator(e["params"], depth, width, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    x = torch.as_tensor(np.random.default_rng(7).uniform(-3, 3, (m, d)), dtype=s.dtype, device="cuda")
    ll_ref, g_ref = s.grad_loglike(x)
    for _ in range(2):
        ll, g = _call(s, x, m)
        assert torch.equal(ll, ll_ref) and torch.equal(g, g_ref)
    s.close()
