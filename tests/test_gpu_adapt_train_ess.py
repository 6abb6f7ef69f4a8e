"""GPU parity of covariance adaptation (Welford + Cholesky + z remap), emulator
training (forward / backward / Adam), the ESS kernel and the autograd.Function."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_common import emulator_case, make_emulator_sampler, rel_err, whitening

pytestmark = pytest.mark.gpu


def _small(prec, n=128, d=6, **kw):
    e = emulator_case(d, 256, 2, out_s=6.0, out_m=20.0)
    mu, L = whitening(d, 2, scale=0.5)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    theta0 = np.clip(mu + np.random.default_rng(1).normal(size=(n, d)) @ L.T, -2.9, 2.9)
    s = make_emulator_sampler(prec, e, n, mu=mu, L=L, lower=lower, upper=upper, theta0=theta0, **kw)
    return s, e, mu, L, lower, upper


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adapt_cov_from_external_samples(prec):
    s, e, mu, L, lo, up = _small(prec)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 6))
    x = rng.normal(size=(5000, 6)) @ A.T * 0.2 + 0.5
    s.welford_reset()
    s.welford_add(torch.as_tensor(x[:1700]))
    s.welford_add(torch.as_tensor(x[1700:]))
    st0 = s.get_state()
    mu_n, L_n, used = s.adapt_cov()
    xs = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
    mref, cref = O.pooled_cov(xs)
    rc, Lref, uref = O.cholesky_jitter(cref)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert used == 0.0 and rc == 0
    assert np.allclose(mu_n, mref, rtol=tol, atol=tol) and np.allclose(L_n, Lref, rtol=1e-9 if prec == "fp64" else 1e-5, atol=1e-9)
    # chain x unchanged by the remap, log pi re-evaluated under the new whitening
    st1 = s.get_state()
    x0 = mu + st0["z"] @ L.T
    x1 = mu_n + st1["z"] @ L_n.T
    assert np.allclose(x0, x1, atol=1e-10 if prec == "fp64" else 2e-5)
    m = O.Model(6, emulator=e, lower=lo, upper=up, mu=mu_n, L=L_n)
    rl, _ = m.logpost(st1["z"])
    fin = np.isfinite(rl)
    assert np.max(np.abs(st1["logp"][fin] - rl[fin]) / np.maximum(1, np.abs(rl[fin]))) < (1e-10 if prec == "fp64" else 1e-5)
    s.close()


def test_adapt_cov_inside_steps_matches_recorded_samples():
    s, *_ = _small("fp64", n=160)
    s.welford_reset()
    out = torch.empty((40, 160, 6), dtype=torch.float64, device="cuda")
    s.step("mala", 40, eps=0.3, samples=out)
    mu_n, L_n, used = s.adapt_cov()
    x = out.cpu().numpy().reshape(-1, 6)
    assert np.allclose(mu_n, x.mean(axis=0), rtol=1e-10, atol=1e-12)
    assert np.allclose(L_n @ L_n.T, np.cov(x.T), rtol=1e-9, atol=1e-12)
    s.close()


def test_adapt_cov_errors():
    from paper_2606_04895_gb300 import BstError
    s, *_ = _small("fp64")
    s.welford_reset()
    with pytest.raises(BstError, match="ERR_STATE"):
        s.adapt_cov()
    s.welford_add(torch.zeros((10, 6), dtype=torch.float64))  # zero covariance
    with pytest.raises(BstError, match="ERR_NOT_PD"):
        s.adapt_cov()
    # rank-deficient (fewer samples than dims): rescued by the diagonal loading
    s.welford_reset()
    s.welford_add(torch.as_tensor(np.random.default_rng(0).normal(size=(4, 6))))
    mu_n, L_n, used = s.adapt_cov(1e-10)
    assert used > 0
    s.close()


def test_training_gradient_matches_oracle():
    from paper_2606_04895_gb300 import Sampler
    d, D, w = 8, 3, 256
    e = S.emulator(d, width=w, depth=D, seed=3, out_m=200.0, out_s=50.0)
    s = Sampler(d, 8, precision="fp32", likelihood="emulator")
    s.set_emulator(e["params"], D, w, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    X = np.random.default_rng(0).uniform(-3, 3, (777, d))
    y = 200 + 50 * np.random.default_rng(1).normal(size=777)
    loss, g = s.train_grad(torch.as_tensor(X, dtype=torch.float32, device="cuda"),
                           torch.as_tensor(y, dtype=torch.float32, device="cuda"))
    Xf = X.astype(np.float32).astype(np.float64)
    yf = y.astype(np.float32).astype(np.float64)
    Pf = e["params"].astype(np.float32).astype(np.float64)
    lref, gref = O.train_loss_grad(d, D, w, Pf, e["in_m"], e["in_s"], e["out_m"], e["out_s"], Xf, yf)
    assert abs(loss.item() - lref) / lref < 1e-4
    assert rel_err(g.cpu().numpy(), gref) < 1e-3
    s.close()


def test_training_gradient_log_output_matches_oracle():
    """Log output (regression target log(chi2 - floor), standardised): loss and parameter gradient
    of bst_train_grad against the FP64 oracle on the FP32-rounded inputs."""
    from paper_2606_04895_gb300 import Sampler
    d, D, w = 8, 3, 256
    e = S.emulator(d, width=w, depth=D, seed=3, out_m=3.0, out_s=1.5, out_log=1, out_floor=240.0)
    s = Sampler(d, 8, precision="fp32", likelihood="emulator")
    s.set_emulator(e["params"], D, w, e["in_m"], e["in_s"], e["out_m"], e["out_s"], out_log=1,
                   out_floor=e["out_floor"])
    X = np.random.default_rng(0).uniform(-3, 3, (777, d))
    y = 241.0 + np.exp(3.0 + 1.5 * np.random.default_rng(1).normal(size=777))
    loss, g = s.train_grad(torch.as_tensor(X, dtype=torch.float32, device="cuda"),
                           torch.as_tensor(y, dtype=torch.float32, device="cuda"))
    Xf = X.astype(np.float32).astype(np.float64)
    yf = y.astype(np.float32).astype(np.float64)
    Pf = e["params"].astype(np.float32).astype(np.float64)
    lref, gref = O.train_loss_grad(d, D, w, Pf, e["in_m"], e["in_s"], e["out_m"], e["out_s"], Xf, yf,
                                   out_log=1, out_floor=e["out_floor"])
    assert abs(loss.item() - lref) / lref < 1e-4
    assert rel_err(g.cpu().numpy(), gref) < 1e-3
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("out_log", [0, 1])
def test_tensor_core_training_gradient_matches_oracle(prec, out_log):
    """Handles of a tensor-core precision train the hidden layers on tcgen05 (BF16 operands,
    FP32 accumulation; 8-512x4-1, batch 1024 = two 512-row multiples): loss and gradient against
    the oracle's BF16 mixed-precision training mode (operands of the hidden-layer products rounded
    at the same points) on the FP32-rounded inputs."""
    from paper_2606_04895_gb300 import Sampler
    d, D, w, m = 8, 4, 512, 1024
    kw = dict(out_log=1, out_floor=240.0) if out_log else {}
    om, osd = (3.0, 1.5) if out_log else (200.0, 50.0)
    e = S.emulator(d, width=w, depth=D, seed=3, out_m=om, out_s=osd, **kw)
    s = Sampler(d, 8, precision=prec, likelihood="emulator")
    s.set_emulator(e["params"], D, w, e["in_m"], e["in_s"], e["out_m"], e["out_s"], **kw)
    X = np.random.default_rng(0).uniform(-3, 3, (m, d))
    rng = np.random.default_rng(1)
    y = 241.0 + np.exp(3.0 + 1.5 * rng.normal(size=m)) if out_log else 200 + 50 * rng.normal(size=m)
    loss, g = s.train_grad(torch.as_tensor(X, dtype=torch.float32, device="cuda"),
                           torch.as_tensor(y, dtype=torch.float32, device="cuda"))
    Xf = X.astype(np.float32).astype(np.float64)
    yf = y.astype(np.float32).astype(np.float64)
    Pf = e["params"].astype(np.float32).astype(np.float64)
    lref, gref = O.train_loss_grad(d, D, w, Pf, e["in_m"], e["in_s"], e["out_m"], e["out_s"], Xf, yf,
                                   bf16=True, **kw)
    assert abs(loss.item() - lref) / lref < 1e-4
    assert rel_err(g.cpu().numpy(), gref) < 3e-3, rel_err(g.cpu().numpy(), gref)
    # and it is not the FP32 gradient: the BF16 rounding of the operands is visible
    _, g64 = O.train_loss_grad(d, D, w, Pf, e["in_m"], e["in_s"], e["out_m"], e["out_s"], Xf, yf, **kw)
    assert rel_err(gref, g64) > 1e-4
    s.close()


def test_tensor_core_training_reduces_loss():
    """Adam on a BF16 handle (tensor-core training): the loss falls on a smooth target and the
    sampling weights follow the master weights."""
    from paper_2606_04895_gb300 import Sampler
    d, D, w = 4, 3, 256
    e = S.emulator(d, width=w, depth=D, seed=3, out_m=10.0, out_s=5.0)
    s = Sampler(d, 8, precision="bf16", likelihood="emulator")
    s.set_emulator(e["params"], D, w, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    X = torch.as_tensor(np.random.default_rng(0).uniform(-3, 3, (2048, d)), dtype=torch.float32, device="cuda")
    y = (X ** 2).sum(dim=1) * 2.0
    loss = torch.zeros(1, device="cuda")
    losses = []
    for it in range(200):
        s.train_step(X, y, lr=3e-3, loss_out=loss)
        losses.append(loss.item())
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    s.close()


def test_training_reduces_loss_and_updates_sampling_weights():
    from paper_2606_04895_gb300 import Sampler
    d, D, w = 4, 2, 256
    e = S.emulator(d, width=w, depth=D, seed=3, out_m=10.0, out_s=5.0)
    s = Sampler(d, 8, precision="fp32", likelihood="emulator")
    s.set_emulator(e["params"], D, w, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    X = torch.as_tensor(np.random.default_rng(0).uniform(-3, 3, (2048, d)), dtype=torch.float32, device="cuda")
    y = (X ** 2).sum(dim=1) * 2.0
    loss = torch.zeros(1, device="cuda")
    losses = []
    for it in range(200):
        s.train_step(X, y, lr=3e-3, loss_out=loss)
        losses.append(loss.item())
    assert losses[-1] < 0.1 * losses[0]
    P = s.get_emulator()
    ref = O.Model(d, emulator=dict(e, params=P))
    x = np.random.default_rng(5).uniform(-2, 2, (33, d))
    rl, rg = ref.loglike(x)
    ll, g = s.grad_loglike(x)
    assert np.max(np.abs(ll.double().cpu().numpy() - rl) / np.maximum(1, np.abs(rl))) < 1e-5
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ess_matches_oracle(prec):
    s, *_ = _small(prec, n=64)
    rng = np.random.default_rng(0)
    n = 600
    phi = np.linspace(0.1, 0.9, 6)
    x = np.zeros((n, 64, 6))
    x[0] = rng.normal(size=(64, 6))
    for t in range(1, n):
        x[t] = phi * x[t - 1] + rng.normal(size=(64, 6))
    xt = torch.as_tensor(x, dtype=s.dtype, device="cuda")
    ess = s.ess(xt)
    ref = O.ess(xt.double().cpu().numpy())
    assert np.allclose(ess, ref, rtol=1e-9 if prec == "fp64" else 1e-4)
    s.close()


def test_autograd_function_gradient():
    from paper_2606_04895_gb300 import emulator_logl
    s, e, *_ = _small("fp64", n=8)
    th = torch.tensor(np.random.default_rng(2).uniform(-2, 2, (5, 6)), dtype=torch.float64, device="cuda",
                      requires_grad=True)
    w = torch.arange(1, 6, dtype=torch.float64, device="cuda")
    (emulator_logl(th, s) * w).sum().backward()
    ref = O.Model(6, emulator=e)
    _, rg = ref.loglike(th.detach().cpu().numpy())
    assert np.allclose(th.grad.cpu().numpy(), rg * w.cpu().numpy()[:, None], rtol=1e-9, atol=1e-12)
    # central finite differences through the forward op
    h = 1e-5
    x0 = th.detach().clone()
    for i in range(6):
        dx = torch.zeros_like(x0); dx[:, i] = h
        fd = (s.loglike(x0 + dx) - s.loglike(x0 - dx)) / (2 * h)
        assert np.allclose(fd.cpu().numpy(), rg[:, i], rtol=1e-6, atol=1e-8)
    s.close()


def test_welford_stats_and_rank_order_merge():
    """Two handles standing in for two ranks: merging their statistics in rank order
    reproduces the pooled covariance of all samples (numpy.cov)."""
    sa, *_ = _small("fp64")
    sb, *_ = _small("fp64")
    rng = np.random.default_rng(8)
    xa = rng.normal(size=(700, 6)) * 0.3 + 1.0
    xb = rng.normal(size=(500, 6)) * 0.5 - 0.5
    for s, x in ((sa, xa), (sb, xb)):
        s.welford_reset()
        s.welford_add(torch.as_tensor(x))
    na, ma, Ma = sa.welford_stats()
    nb, mb, Mb = sb.welford_stats()
    assert na == 700 and np.allclose(ma, xa.mean(axis=0), rtol=1e-12)
    assert np.allclose(Ma / (na - 1), np.cov(xa.T), rtol=1e-10)
    for s in (sa, sb):
        s.welford_reset()
        s.welford_merge(na, ma, Ma)
        s.welford_merge(nb, mb, Mb)
    mu_a, L_a, _ = sa.adapt_cov()
    mu_b, L_b, _ = sb.adapt_cov()
    allx = np.concatenate([xa, xb])
    assert np.array_equal(mu_a, mu_b) and np.array_equal(L_a, L_b)
    assert np.allclose(mu_a, allx.mean(axis=0), rtol=1e-12)
    assert np.allclose(L_a @ L_a.T, np.cov(allx.T), rtol=1e-9)
    sa.close(); sb.close()


def test_train_apply_equals_train_step():
    from paper_2606_04895_gb300 import Sampler
    d, D, w = 4, 2, 256
    e = S.emulator(d, width=w, depth=D, seed=3, out_m=10.0, out_s=5.0)
    X = torch.as_tensor(np.random.default_rng(0).uniform(-3, 3, (1024, d)), dtype=torch.float32, device="cuda")
    y = (X ** 2).sum(dim=1)
    a = Sampler(d, 8, precision="fp32", likelihood="emulator")
    b = Sampler(d, 8, precision="fp32", likelihood="emulator")
    for s in (a, b):
        s.set_emulator(e["params"], D, w, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    for _ in range(3):
        a.train_step(X, y, lr=1e-3)
        _, g = b.train_grad(X, y)
        b.train_apply(g, lr=1e-3)
    assert np.array_equal(a.get_emulator(), b.get_emulator())
    a.close(); b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_r_minus_1_worked_example(prec):
    """The hand-worked one-dimensional case of the oracle pins through the device path:
    chains (0, 2) and (4, 6) give R - 1 = B / W = 8 / 2 = 4."""
    from paper_2606_04895_gb300 import Sampler
    s = Sampler(1, 2, precision=prec, likelihood="emulator")
    x = torch.tensor([[[0.0], [4.0]], [[2.0], [6.0]]], dtype=s.dtype, device="cuda")
    assert s.r_minus_1(x) == pytest.approx(4.0, rel=1e-12)
    s.close()


@pytest.mark.parametrize("prec,n_chains,d", [("fp64", 64, 6), ("fp32", 64, 6), ("fp32", 200, 27), ("fp64", 33, 27),
                                             ("bf16", 300, 8)])
def test_r_minus_1_matches_oracle(prec, n_chains, d):
    """R - 1 of AR(1) chains with chain-dependent offsets (ragged chain counts: the device
    blocks hold 32 chains) against the FP64 oracle on the same working-precision draws."""
    from paper_2606_04895_gb300 import Sampler
    s = Sampler(d, n_chains, precision=prec, likelihood="emulator")
    rng = np.random.default_rng(4)
    n = 300
    A = rng.normal(size=(d, d)) / np.sqrt(d) + np.eye(d)
    x = np.zeros((n, n_chains, d))
    x[0] = rng.normal(size=(n_chains, d))
    for t in range(1, n):
        x[t] = 0.7 * x[t - 1] + rng.normal(size=(n_chains, d))
    x = x @ A.T + 0.3 * rng.normal(size=(1, n_chains, d))
    xt = torch.as_tensor(x, dtype=s.dtype, device="cuda")
    r = s.r_minus_1(xt)
    ref = O.r_minus_1(xt.double().cpu().numpy())
    assert np.isfinite(ref) and ref > 0
    assert r == pytest.approx(ref, rel=1e-8)
    s.close()


def test_r_minus_1_undefined_is_nan():
    from paper_2606_04895_gb300 import Sampler
    s = Sampler(3, 40, precision="fp32", likelihood="emulator")
    x = torch.randn(50, 40, 3, device="cuda")
    x[:, :, 1] = 2.0  # no spread in one dimension: B_11 = 0
    assert np.isnan(s.r_minus_1(x))
    s.close()


@pytest.mark.parametrize("prec,n_chains,d,n_draws", [("fp32", 64, 6, 301), ("fp64", 33, 27, 120), ("bf16", 300, 8, 77),
                                                      ("fp32", 16384, 27, 40)])
def test_quantiles_match_oracle(prec, n_chains, d, n_draws):
    """Exact order statistics (radix select) against numpy's on the same working-precision
    draws: negative values, ties (a coarse grid in one dimension), the extreme levels 0 and 1."""
    from paper_2606_04895_gb300 import Sampler
    s = Sampler(d, n_chains, precision=prec, likelihood="emulator")
    rng = np.random.default_rng(7)
    x = rng.normal(size=(n_draws, n_chains, d)) * np.linspace(0.1, 3.0, d) - 0.5
    x[:, :, 0] = np.round(x[:, :, 0] * 4) / 4  # many ties
    xt = torch.as_tensor(x, dtype=s.dtype, device="cuda")
    q = [0.0, 0.025, 0.16, 0.5, 0.84, 0.975, 1.0]
    out = s.quantiles(xt, q)
    ref = O.quantiles(xt.double().cpu().numpy(), q)
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-12)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_credible_metric_matches_oracle(prec):
    from paper_2606_04895_gb300 import Sampler
    d, n_chains, n = 5, 96, 200
    s = Sampler(d, n_chains, precision=prec, likelihood="emulator")
    x = np.random.default_rng(8).normal(size=(n, n_chains, d)) * 2.0 + 1.0
    xt = torch.as_tensor(x, dtype=s.dtype, device="cuda")
    lo0, hi0 = np.full(d, 1.0 - 2.0), np.full(d, 1.0 + 2.0)  # the true 68 % limits, about +-1 sd
    for alpha in (0.68, 0.95):
        cm = s.credible_metric(xt, alpha, lo0, hi0)
        ref = O.credible_metric(xt.double().cpu().numpy(), alpha, lo0, hi0)
        assert np.allclose(cm, ref, rtol=1e-10, atol=1e-12)
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 2e-5)])
def test_set_whitening_keeps_x_and_shifts_log_pi_by_log_det(prec, tol):
    """A new whitening keeps every chain's x; log pi_z changes by log|det L_new| - log|det L_old|
    (Algorithm 1), and grad_z by L_new^T L_old^-T."""
    from paper_2606_04895_gb300 import BstError
    s, e, mu, L, lo, up = _small(prec, n=96)
    st0 = s.get_state()
    x0 = mu + st0["z"] @ L.T
    rng = np.random.default_rng(11)
    mu2 = mu + 0.05 * rng.normal(size=mu.size)
    L2 = np.tril(0.3 * rng.normal(size=L.shape)) + np.diag(np.full(mu.size, 0.6))
    s.set_whitening(mu2, L2)
    st1 = s.get_state()
    m, Lw = s.whitening()
    assert np.allclose(m, mu2) and np.allclose(Lw, L2)
    x1 = mu2 + st1["z"] @ L2.T
    assert np.max(np.abs(x1 - x0)) < tol * 10
    fin = np.isfinite(st0["logp"])
    dld = np.sum(np.log(np.diag(L2))) - np.sum(np.log(np.diag(L)))
    assert np.allclose(st1["logp"][fin] - st0["logp"][fin], dld, rtol=0, atol=tol * max(1.0, np.abs(st0["logp"]).max()))
    gx = np.linalg.solve(L.T, st0["grad"].T).T  # grad_x = L^-T grad_z
    assert np.allclose(st1["grad"][fin], (gx @ L2)[fin], rtol=0, atol=tol * 10 * max(1.0, np.abs(gx @ L2).max()))
    # step multipliers are the whitening L diag(m)
    s.set_step_multipliers(np.arange(1, mu.size + 1))
    assert np.allclose(s.whitening()[1], L2 * np.arange(1, mu.size + 1)[None, :])
    with pytest.raises(BstError):
        s.set_whitening(mu2, np.zeros_like(L2))
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_draw_positions_match_oracle(prec):
    """Initial positions of the three strategies of Sec. 3.1 drawn on the device against the
    oracle's draws from the same Philox streams (uniform draws bit for bit; Gaussian to
    rounding of the Box-Muller transcendentals), then usable by init_chains."""
    from paper_2606_04895_gb300 import BstError, Sampler
    d, n, seed = 5, 300, 21
    s = Sampler(d, n, precision=prec, likelihood="emulator", seed=seed)
    c = np.array([0.3, -0.2, 1.0, 0.0, -1.5])
    lo, hi = np.full(d, -3.0), np.array([3.0, 2.0, 3.0, 1.0, 0.5])
    Lc = np.tril(np.random.default_rng(2).normal(size=(d, d))) * 0.3 + 0.5 * np.eye(d)
    rep = s.draw_positions("repeated", center=c)
    assert np.array_equal(rep, np.tile(c, (n, 1)))
    u = s.draw_positions("uniform", lower=lo, upper=hi)
    assert np.array_equal(u, O.draw_positions(O.INIT_UNIFORM, seed, n, d, lower=lo, upper=hi))
    g = s.draw_positions("gaussian", center=c, L=Lc)
    ref = O.draw_positions(O.INIT_GAUSSIAN, seed, n, d, center=c, Lc=Lc)
    assert np.max(np.abs(g - ref)) < 1e-12
    with pytest.raises(BstError):
        s.draw_positions("uniform", lower=hi, upper=lo)
    s.close()


def test_burn_in_driver_adapts_whitening_and_step_size():
    """The burn-in driver on the library: two adaptation iterations change the whitening, and
    the adapted step size gives an acceptance statistic near the 0.65 target."""
    from paper_2606_04895_gb300 import driver
    s, e, mu, L, lo, up = _small("fp32", n=128)
    _, L0 = s.whitening()
    eps, hist = driver.burn_in(s, "mala", eps0=0.2, n_iter=2, adapt_steps=200, chunk=40, cov_steps=200)
    _, L1 = s.whitening()
    assert np.isfinite(eps) and eps > 0 and len(hist) == 2
    assert not np.allclose(L1, L0)
    st = s.step("mala", 200, eps=eps)
    assert 0.3 < st["accept_stat"] < 0.95, st
    s.close()


@pytest.mark.parametrize("prec,n_chains,d,n_draws,n_ref,n_proj", [
    ("fp32", 64, 6, 31, 1000, 64),   # unequal sizes
    ("fp64", 33, 27, 20, 660, 37),   # equal sizes, 27-D
    ("fp32", 40, 1, 5, 77, 7),       # d = 1: projections +-x, many ties within and across the sets
    ("fp64", 3, 2, 1, 1, 5),         # three draws against one reference point
])
def test_sliced_wasserstein_matches_oracle(prec, n_chains, d, n_draws, n_ref, n_proj):
    """Sliced Wasserstein distance (Sec. 4.1) against the oracle on the same working-precision
    values: the device integrates |F_a - F_b| over x on the merged sorted projections, the
    oracle |F^-1 - G^-1| over t."""
    from paper_2606_04895_gb300 import Sampler
    s = Sampler(d, n_chains, precision=prec, likelihood="emulator")
    rng = np.random.default_rng(12)
    x = rng.normal(size=(n_draws, n_chains, d)) * np.linspace(0.5, 2.0, d)
    r = rng.standard_t(5, size=(n_ref, d)) + 0.3
    if d == 1:
        x, r = np.round(x * 2) / 2, np.round(r * 2) / 2
    xt = torch.as_tensor(x, dtype=s.dtype, device="cuda")
    rt = torch.as_tensor(r, dtype=s.dtype, device="cuda")
    got = s.sliced_wasserstein(xt, rt, n_proj=n_proj, seed=5)
    ref = O.sliced_wasserstein(xt.double().cpu().numpy().reshape(-1, d), rt.double().cpu().numpy(), n_proj=n_proj,
                               seed=5)
    assert ref > 0
    assert got == pytest.approx(ref, rel=1e-9)
    assert s.sliced_wasserstein(xt, xt.reshape(-1, d).flip(0).contiguous(), n_proj=n_proj, seed=5) == 0.0
    s.close()


def test_sliced_wasserstein_of_a_shift_over_several_sorting_chunks():
    """60,000 projected values per direction and 3,000 directions exceed one sorting chunk
    (2^27 values): the distance between a set and its shift by c is mean_k |c . u_k| exactly,
    u_k the oracle's directions."""
    from paper_2606_04895_gb300 import Sampler
    d, n_chains, n_draws = 5, 1000, 30
    s = Sampler(d, n_chains, precision="fp64", likelihood="emulator")
    rng = np.random.default_rng(13)
    x = rng.normal(size=(n_draws, n_chains, d))
    c = np.array([0.5, -1.0, 0.25, 2.0, 0.0])
    xt = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.as_tensor(x.reshape(-1, d) + c, dtype=torch.float64, device="cuda")
    got = s.sliced_wasserstein(xt, qt, n_proj=3000, seed=3)
    U = O.swd_directions(3, 3000, d)
    assert got == pytest.approx(float(np.mean(np.abs(U @ c))), rel=1e-10)
    s.close()


def test_sliced_wasserstein_rejects_bad_arguments():
    from paper_2606_04895_gb300 import BstError, Sampler
    s = Sampler(3, 8, precision="fp32", likelihood="emulator")
    x = torch.zeros(2, 8, 3, device="cuda")
    with pytest.raises(BstError):
        s.sliced_wasserstein(x, torch.zeros(4, 3, device="cuda"), n_proj=0)
    with pytest.raises(BstError):
        s.sliced_wasserstein(x, torch.zeros(4, 2, device="cuda"))
    s.close()


def test_sliced_wasserstein_at_the_comparison_scale():
    """The comparison scale of Sec. 4.1 (500 directions, 100,000 reference points) with 100 draws
    of 1,000 chains of a 27-D target in FP32: a set against its shift by c gives mean_k |c . u_k|."""
    from paper_2606_04895_gb300 import Sampler
    d, n_chains, n_draws = 27, 1000, 100
    s = Sampler(d, n_chains, precision="fp32", likelihood="emulator")
    g = torch.Generator(device="cuda")
    g.manual_seed(14)
    xt = torch.randn((n_draws, n_chains, d), generator=g, device="cuda")
    c = np.linspace(-1.0, 1.0, d)
    qt = (xt.reshape(-1, d) + torch.as_tensor(c, dtype=torch.float32, device="cuda")).contiguous()
    got = s.sliced_wasserstein(xt, qt, n_proj=500, seed=0)
    U = O.swd_directions(0, 500, d)
    assert got == pytest.approx(float(np.mean(np.abs(U @ c))), rel=2e-5)
    s.close()
