"""Pins for the oracle's likelihoods and whitened target.

Each check is independent of the oracle's own arithmetic: a closed form
(least-squares quadratic form of the linear theory map), a special case
(zero-noise truth, zero weights, odd symmetry), central finite differences,
torch autograd on a separately built network, or the log-determinant identity
of the whitened density (paper Sec. 2.2, Eq. (2.12))."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S


def _fd_grad(f, x, h=1e-5):
    g = np.zeros_like(x)
    for i in range(x.size):
        e = np.zeros_like(x); e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def _analytic_model(t, **kw):
    return O.Model(t["d"], lik="analytic", analytic=t, lower=t["lower"], upper=t["upper"],
                   gauss=t["gauss"], **kw)


def test_linear_theory_map_is_exact_quadratic():
    t = S.target(6, linear=True, seed=0)
    m = _analytic_model(t)
    J = t["A"] @ t["B"]
    y = t["data"] - t["A"] @ t["c"]
    xhat, res, *_ = np.linalg.lstsq(J, y, rcond=None)
    chi2_min = float(res[0])
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = xhat + 0.05 * rng.standard_normal(6)
        dx = x - xhat
        expect = -0.5 * (chi2_min + dx @ (J.T @ J) @ dx) / t["sigma"] ** 2
        got = m.loglike(x)[0][0]
        assert got == pytest.approx(expect, rel=1e-10, abs=1e-9)


def test_truth_residual_is_the_drawn_noise():
    """data = f(theta*) + sigma xi (numpy matmuls in the input recipe), so the
    oracle's logL(theta*) must be exactly -|xi|^2 / 2 for every target shape."""
    for kw in ({"d": 6}, {"d": 8}, {"d": 27, "nuisance": True}, {"d": 6, "linear": True}):
        seed = 3
        t = S.target(seed=seed, **kw)
        m = _analytic_model(t)
        xi = np.random.default_rng(seed + 2).standard_normal(t["data"].size)
        assert m.loglike(t["theta_star"], grad=False)[0] == pytest.approx(-0.5 * xi @ xi, rel=1e-10)


@pytest.mark.parametrize("kind", ["tanh6", "linear6", "sterile8", "nuis27"])
def test_analytic_gradient_finite_differences(kind):
    kw = {"tanh6": dict(d=6), "linear6": dict(d=6, linear=True), "sterile8": dict(d=8),
          "nuis27": dict(d=27, nuisance=True)}[kind]
    t = S.target(seed=11, **kw)
    m = _analytic_model(t)
    rng = np.random.default_rng(2)
    for _ in range(3):
        x = t["theta_star"] + 0.2 * rng.standard_normal(t["d"])
        lp, g = m.loglike(x)
        fd = _fd_grad(lambda v: m.loglike(v, grad=False)[0], x, h=1e-5)
        assert np.allclose(g[0], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def _torch_emulator(e, x, bf16=False, fp16=False):
    W, b, wo, bo = S.unpack_emulator(e)
    r = ((lambda t: t.to(torch.bfloat16).to(torch.float64)) if bf16 else
         (lambda t: t.to(torch.float16).to(torch.float64)) if fp16 else (lambda t: t))
    X = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    u = (X - torch.tensor(e["in_m"])) / torch.tensor(e["in_s"])
    h = torch.tanh(u @ torch.tensor(W[0]).T + torch.tensor(b[0]))
    for l in range(1, len(W)):
        h = torch.tanh(r(h) @ r(torch.tensor(W[l])).T + torch.tensor(b[l]))
    out = h @ torch.tensor(wo) + bo
    logl = -0.5 * (e["out_s"] * out + e["out_m"])
    return logl, X


@pytest.mark.parametrize("d,width,depth", [(6, 32, 1), (8, 64, 4), (27, 48, 3)])
def test_emulator_matches_torch_autograd(d, width, depth):
    e = S.emulator(d, width=width, depth=depth, seed=4, out_m=3.0, out_s=2.5)
    m = O.Model(d, emulator=e)
    x = np.random.default_rng(0).uniform(-2, 2, (7, d))
    lp, g = m.loglike(x)
    logl, X = _torch_emulator(e, x)
    (gt,) = torch.autograd.grad(logl.sum(), X)
    assert np.allclose(lp, logl.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(g, gt.numpy(), rtol=1e-10, atol=1e-12)


def test_emulator_gradient_finite_differences():
    e = S.emulator(8, width=64, depth=4, seed=9, out_s=3.0)
    m = O.Model(8, emulator=e)
    x = np.random.default_rng(5).uniform(-2, 2, 8)
    _, g = m.loglike(x)
    fd = _fd_grad(lambda v: m.loglike(v, grad=False)[0], x)
    assert np.allclose(g[0], fd, rtol=1e-6, atol=1e-8)


def test_emulator_special_cases():
    d, w, D = 6, 16, 3
    e = S.emulator(d, width=w, depth=D, seed=1)
    W, b, wo, bo = S.unpack_emulator(e)
    # all weights zero: out = wo . tanh(b_D) + bo, constant, zero gradient
    Wz = [np.zeros_like(Wl) for Wl in W]
    ez = dict(e, params=S.pack_emulator(Wz, b, wo, 0.7))
    mz = O.Model(d, emulator=ez)
    lp, g = mz.loglike(np.random.default_rng(0).normal(size=(3, d)))
    expect = -0.5 * (e["out_s"] * (wo @ np.tanh(b[-1]) + 0.7) + e["out_m"])
    assert np.allclose(lp, expect, rtol=1e-14) and np.all(g == 0)
    # zero biases: out - bo is odd in u (tanh is odd)
    bz = [np.zeros_like(bl) for bl in b]
    eo = dict(e, params=S.pack_emulator(W, bz, wo, 0.0), out_m=0.0, out_s=1.0)
    mo = O.Model(d, emulator=eo)
    x = np.random.default_rng(1).normal(size=(4, d))
    assert np.allclose(mo.loglike(x, grad=False), -mo.loglike(-x, grad=False), rtol=1e-13)


def test_emulator_bf16_mode_matches_torch_rounding():
    e = S.emulator(8, width=64, depth=4, seed=2, out_s=4.0)
    mb = O.Model(8, emulator=e, bf16=True)
    m = O.Model(8, emulator=e)
    x = np.random.default_rng(3).uniform(-2, 2, (5, 8))
    lpb = mb.loglike(x, grad=False)
    logl, _ = _torch_emulator(e, x, bf16=True)
    assert np.allclose(lpb, logl.detach().numpy(), rtol=1e-12, atol=1e-12)
    # and BF16 differs from FP64 by a BF16-sized amount, not zero, not O(1)
    diff = np.abs(lpb - m.loglike(x, grad=False))
    assert np.all(diff > 0) and np.all(diff < 0.05 * e["out_s"])


def test_emulator_fp16_mode_matches_torch_rounding():
    """FP16 mode: hidden-product operands rounded to binary16 (torch's float16 conversion of the
    FP64 values); logL equals the torch expression, and the gradient equals the BF16-free FP64
    gradient to FP16 accuracy (the adjoint vectors are rounded too)."""
    e = S.emulator(8, width=64, depth=4, seed=2, out_s=4.0)
    mf = O.Model(8, emulator=e, fp16=True)
    m = O.Model(8, emulator=e)
    x = np.random.default_rng(3).uniform(-2, 2, (5, 8))
    lpf, gf = mf.loglike(x)
    logl, _ = _torch_emulator(e, x, fp16=True)
    assert np.allclose(lpf, logl.detach().numpy(), rtol=1e-12, atol=1e-12)
    lp, g = m.loglike(x)
    diff = np.abs(lpf - lp)
    mb = O.Model(8, emulator=e, bf16=True)
    diff_b = np.abs(mb.loglike(x, grad=False) - lp)
    # FP16 keeps three more bits than BF16: its error is several times smaller
    assert np.all(diff > 0) and diff.max() < 0.25 * diff_b.max()
    assert np.max(np.abs(gf - g)) < 5e-3 * np.max(np.abs(g))


def test_emulator_fp16_mode_gradient_scale_is_out_s():
    """The FP16 mode seeds the adjoint without out_s and scales the input gradient by out_s, so the
    gradient is out_s times that of out_s = 1 (same roundings) and stays finite at an out_s whose
    seed would overflow binary16 (65504) if out_s were inside it."""
    e1 = S.emulator(6, width=32, depth=2, seed=7, out_s=1.0)
    eb = dict(e1, out_s=3.0e7)
    x = np.random.default_rng(0).uniform(-1, 1, (4, 6))
    _, g1 = O.Model(6, emulator=e1, fp16=True).loglike(x)
    _, gb = O.Model(6, emulator=eb, fp16=True).loglike(x)
    assert np.all(np.isfinite(gb))
    assert np.allclose(gb, 3.0e7 * g1, rtol=1e-15, atol=0)


def test_whitened_density_log_det_identity():
    t = S.target(6, seed=0)
    rng = np.random.default_rng(0)
    A = rng.normal(size=(6, 6))
    L = np.linalg.cholesky(A @ A.T / 6 * 0.01 + 0.001 * np.eye(6))
    mu = t["theta_star"]
    m = _analytic_model(t, mu=mu, L=L)
    mx = _analytic_model(t)
    z = rng.normal(size=(10, 6))
    lpz, gz = m.logpost(z)
    x = mu + z @ L.T
    lpx, gx = mx.logpost(x)
    assert np.allclose(lpz - lpx, np.sum(np.log(np.diag(L))), rtol=0, atol=1e-9)
    # chain rule: grad_z = L^T grad_x
    assert np.allclose(gz, gx @ L, rtol=1e-10, atol=1e-8)
    # outside the box the density is zero
    zo = np.linalg.solve(L, np.full(6, 3.5) - mu)
    assert m.logpost(zo[None], grad=False)[0] == -np.inf


def test_gaussian_nuisance_prior_term():
    t = S.target(27, nuisance=True, seed=1)
    m = _analytic_model(t)
    x = t["theta_star"] + 0.01
    lp, g = m.logpost(x[None])
    ll, gl = m.loglike(x[None])
    assert lp[0] - ll[0] == pytest.approx(-0.5 * np.sum(x[6:] ** 2), rel=1e-12)
    assert np.allclose(g[0, 6:] - gl[0, 6:], -x[6:], rtol=1e-12)
    assert np.allclose(g[0, :6], gl[0, :6], rtol=1e-12)


def test_emulator_log_output_gradient_finite_differences():
    """Log output (chi2 = floor + exp(out_s out + out_m)): the returned gradient against
    central differences of the returned logL."""
    e = S.emulator(8, width=64, depth=4, seed=9, out_s=1.5, out_m=2.0, out_log=1, out_floor=250.0)
    m = O.Model(8, emulator=e)
    x = np.random.default_rng(5).uniform(-2, 2, 8)
    _, g = m.loglike(x)
    fd = _fd_grad(lambda v: m.loglike(v, grad=False)[0], x)
    assert np.allclose(g[0], fd, rtol=1e-6, atol=1e-8)


def test_emulator_log_output_matches_torch_autograd():
    """The log output is exp of the linear output's standardised value, shifted by the floor:
    logL_log = -(floor + exp(-2 logL_lin')) / 2 with logL_lin' the linear-output logL at
    out_m, out_s; torch autograd of that expression gives the gradient."""
    d, width, depth = 6, 32, 3
    e = S.emulator(d, width=width, depth=depth, seed=4, out_m=1.0, out_s=0.5, out_log=1, out_floor=-3.0)
    m = O.Model(d, emulator=e)
    x = np.random.default_rng(0).uniform(-2, 2, (7, d))
    lp, g = m.loglike(x)
    lin = dict(e, out_log=0)
    logl_lin, X = _torch_emulator(lin, x)  # -(out_s out + out_m) / 2
    logl = -0.5 * (e["out_floor"] + torch.exp(-2.0 * logl_lin))
    (gt,) = torch.autograd.grad(logl.sum(), X)
    assert np.allclose(lp, logl.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(g, gt.numpy(), rtol=1e-10, atol=1e-12)


def test_emulator_log_output_constant_network():
    """All weights zero: out = wo . tanh(b_D) + bo is constant, so chi2 = floor + exp(out_s out + out_m)
    everywhere and the gradient is zero."""
    d, w, D = 5, 16, 2
    e = S.emulator(d, width=w, depth=D, seed=1, out_m=0.3, out_s=2.0, out_log=1, out_floor=10.0)
    W, b, wo, bo = S.unpack_emulator(e)
    ez = dict(e, params=S.pack_emulator([np.zeros_like(Wl) for Wl in W], b, wo, 0.2))
    lp, g = O.Model(d, emulator=ez).loglike(np.random.default_rng(0).normal(size=(3, d)))
    out = wo @ np.tanh(b[-1]) + 0.2
    assert np.allclose(lp, -0.5 * (10.0 + np.exp(2.0 * out + 0.3)), rtol=1e-14) and np.all(g == 0)
