"""Long-run statistics of the GPU samplers against the closed-form posterior of
the linear theory map (paper Sec. 2 samplers; the linear variant of the
synthetic likelihood makes the posterior exactly Gaussian):
mean and covariance within 5 Monte Carlo standard errors, with the standard
errors taken from the spread of independent chains (ensembles for AIES)."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _closed_form(seed=0, n_data=64):
    t = S.target(6, linear=True, seed=seed, n_data=n_data)
    J = t["A"] @ t["B"]
    y = t["data"] - t["A"] @ t["c"]
    cov = np.linalg.inv(J.T @ J / t["sigma"] ** 2)
    mean = cov @ (J.T @ y) / t["sigma"] ** 2
    return t, mean, cov


def _check(samples, mean, cov, nsig=5.0):
    n, M, d = samples.shape
    cm = samples.mean(axis=0)
    se_m = cm.std(axis=0, ddof=1) / np.sqrt(M)
    zm = (cm.mean(axis=0) - mean) / se_m
    dev = samples - mean
    cc = np.einsum("tca,tcb->cab", dev, dev) / n
    zc = (cc.mean(axis=0) - cov) / (cc.std(axis=0, ddof=1) / np.sqrt(M))
    assert np.all(np.abs(zm) < nsig), zm
    assert np.all(np.abs(zc) < nsig), zc


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kernel,eps,steps,kw", [("mh", 0.6, 3000, {}), ("mala", 0.5, 2000, {}),
                                                 ("hmc", 0.3, 500, {"n_leapfrog": 8}), ("nuts", 0.5, 400, {}),
                                                 ("nuts", 1.2, 800, {}), ("nuts_multinomial", 0.5, 400, {}),
                                                 ("nuts_multinomial", 1.2, 800, {})])
def test_closed_form_moments(prec, kernel, eps, steps, kw):
    from paper_2606_04895_gb300 import Sampler
    t, mean, cov = _closed_form()
    Lp = np.linalg.cholesky(cov)
    n = 256
    s = Sampler(6, n, precision=prec, likelihood="analytic", seed=17)
    s.set_analytic(t["A"], t["B"], t["c"], t["data"], t["sigma"], linear=True)
    theta0 = mean + S.chains_init(n, 6, seed=2) @ Lp.T
    # imperfect whitening on purpose
    s.init_chains(theta0, t["lower"], t["upper"], mu=mean + 0.2 * np.sqrt(np.diag(cov)), L=1.15 * Lp)
    out = torch.empty((steps, n, 6), dtype=s.dtype, device="cuda")
    s.step(kernel, steps, eps=eps, samples=out, **kw)
    x = out.double().cpu().numpy()[steps // 5:]
    _check(x, mean, cov)
    s.close()


@pytest.mark.parametrize("kernel", ["aies", "aies_de"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_aies_closed_form_moments(prec, kernel):
    from paper_2606_04895_gb300 import Sampler
    t, mean, cov = _closed_form()
    Lp = np.linalg.cholesky(cov)
    n_ens = 32
    n = 64 * n_ens
    s = Sampler(6, n, precision=prec, likelihood="analytic", seed=5)
    s.set_analytic(t["A"], t["B"], t["c"], t["data"], t["sigma"], linear=True)
    theta0 = mean + S.chains_init(n, 6, seed=3) @ Lp.T
    s.init_chains(theta0, t["lower"], t["upper"])
    steps = 1200
    out = torch.empty((steps, n, 6), dtype=s.dtype, device="cuda")
    s.step(kernel, steps, eps=0.1, samples=out)
    x = out.double().cpu().numpy()[steps // 4:]
    ens = x.reshape(x.shape[0], n_ens, 64, 6).transpose(0, 2, 1, 3).reshape(-1, n_ens, 6)
    _check(ens, mean, cov)
    s.close()


def test_bf16_emulator_chains_cover_their_target():
    """BF16 tensor-core MALA on an emulator target: the chains' moments agree with the
    same emulator sampled by the FP64 CUDA-core path (independent chains, same target
    up to BF16 rounding)."""
    from paper_2606_04895_gb300 import Sampler
    d = 8
    e = S.emulator(d, width=256, depth=3, seed=5, out_m=30.0, out_s=6.0)
    res = {}
    for prec in ("bf16", "fp64"):
        n = 1024
        s = Sampler(d, n, precision=prec, likelihood="emulator", seed=23 if prec == "bf16" else 29)
        s.set_emulator(e["params"], 3, 256, e["in_m"], e["in_s"], e["out_m"], e["out_s"])
        th = np.clip(np.random.default_rng(1).normal(size=(n, d)), -2.5, 2.5)
        s.init_chains(th, np.full(d, -3.0), np.full(d, 3.0), L=0.6 * np.eye(d))
        s.step("mala", 500, eps=0.25, stats=False)
        out = torch.empty((1500, n, d), dtype=s.dtype, device="cuda")
        s.step("mala", 1500, eps=0.25, samples=out)
        x = out.double().cpu().numpy()
        cm = x.mean(axis=0)
        res[prec] = (cm.mean(axis=0), cm.std(axis=0, ddof=1) / np.sqrt(n))
        s.close()
    (m1, s1), (m2, s2) = res["bf16"], res["fp64"]
    z = (m1 - m2) / np.sqrt(s1 ** 2 + s2 ** 2)
    assert np.all(np.abs(z) < 5), z


def test_convergence_metrics_on_sampler_output():
    """R - 1 and the credible metric (Sec. 4.1) of MALA draws on the linear target against its
    exact Gaussian posterior: near zero after mixing; R - 1 large for dispersed, unmixed starts."""
    from paper_2606_04895_gb300 import Sampler
    t, mean, cov = _closed_form()
    Lp = np.linalg.cholesky(cov)
    sd = np.sqrt(np.diag(cov))
    n, steps = 256, 2000
    s = Sampler(6, n, precision="fp32", likelihood="analytic", seed=23)
    s.set_analytic(t["A"], t["B"], t["c"], t["data"], t["sigma"], linear=True)
    theta0 = mean + 4.0 * S.chains_init(n, 6, seed=4) @ Lp.T
    s.init_chains(theta0, t["lower"], t["upper"], mu=mean, L=Lp)
    first = torch.empty((3, n, 6), dtype=s.dtype, device="cuda")
    s.step("mala", 3, eps=0.5, samples=first)
    assert s.r_minus_1(first) > 1.0  # three steps from dispersed starts: not mixed
    out = torch.empty((steps, n, 6), dtype=s.dtype, device="cuda")
    s.step("mala", steps, eps=0.5, samples=out)
    x = out[steps // 5:].contiguous()
    assert s.r_minus_1(x) < 0.02
    for alpha, z in ((0.68, 0.994457883), (0.95, 1.959963985)):  # Phi^-1((1 + alpha) / 2)
        cm = s.credible_metric(x, alpha, mean - z * sd, mean + z * sd)
        assert np.all(cm < 0.1), cm
    s.close()


def test_mala_with_step_multipliers_keeps_the_posterior():
    """Per-dimension step multipliers (a larger step on two whitened directions, as the paper
    does for its extension parameters) leave MALA exact: closed-form moments.  (x 2 with
    eps = 0.2: along those directions the posterior spread in the new z is 1/2, so the
    Langevin drift stays stable, eps lambda = 0.8.)"""
    from paper_2606_04895_gb300 import Sampler
    t, mean, cov = _closed_form()
    Lp = np.linalg.cholesky(cov)
    n, steps = 256, 2500
    s = Sampler(6, n, precision="fp32", likelihood="analytic", seed=29)
    s.set_analytic(t["A"], t["B"], t["c"], t["data"], t["sigma"], linear=True)
    s.init_chains(mean + S.chains_init(n, 6, seed=6) @ Lp.T, t["lower"], t["upper"], mu=mean, L=Lp)
    s.set_step_multipliers([1.0, 1.0, 1.0, 1.0, 2.0, 2.0])
    out = torch.empty((steps, n, 6), dtype=s.dtype, device="cuda")
    s.step("mala", steps, eps=0.2, samples=out)
    x = out.double().cpu().numpy()[steps // 5:]
    _check(x, mean, cov)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kernel,eps,steps,kw", [("mala", 0.5, 3000, {}), ("hmc", 0.35, 800, {"n_leapfrog": 6}),
                                                 ("nuts", 0.5, 500, {})])
def test_bounds_penalty_closed_form_marginal_mean(prec, kernel, eps, steps, kw):
    """Smooth bounds (Sec. 3.1): the linear 6-D target with the upper bound of dim 0 at its
    posterior mean and penalty width w = sd_0.  The x_0 marginal is a half-normal of scale sd_0
    joined to one of scale s' = sd_0 w / sqrt(sd_0^2 + w^2), masses in the ratio sd_0 : s', so its
    mean is mu_0 + sqrt(2 / pi) (s' - sd_0); the GPU chains reproduce it within 5 MCSE."""
    from paper_2606_04895_gb300 import Sampler
    t, mean, cov = _closed_form()
    Lp = np.linalg.cholesky(cov)
    sd0 = np.sqrt(cov[0, 0])
    upper = t["upper"].copy()
    upper[0] = mean[0]
    n = 512
    s = Sampler(6, n, precision=prec, likelihood="analytic", seed=23)
    s.set_analytic(t["A"], t["B"], t["c"], t["data"], t["sigma"], linear=True)
    theta0 = mean + S.chains_init(n, 6, seed=2) @ Lp.T
    theta0[:, 0] = np.minimum(theta0[:, 0], mean[0])
    s.init_chains(theta0, t["lower"], upper, mu=mean, L=Lp)
    w = np.zeros(6)
    w[0] = sd0
    s.set_bounds_penalty(w)
    out = torch.empty((steps, n, 6), dtype=s.dtype, device="cuda")
    s.step(kernel, steps, eps=eps, samples=out, **kw)
    x0 = out.double().cpu().numpy()[steps // 5:, :, 0]
    cm = x0.mean(axis=0)
    se = cm.std(ddof=1) / np.sqrt(n)
    sp = sd0 * w[0] / np.sqrt(sd0 ** 2 + w[0] ** 2)
    want = mean[0] + np.sqrt(2.0 / np.pi) * (sp - sd0)
    assert abs(cm.mean() - want) < 5 * se, (cm.mean() - want) / se
    assert abs(cm.mean() - mean[0]) > 10 * se
    s.close()
