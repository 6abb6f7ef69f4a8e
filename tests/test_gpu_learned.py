"""The learned part: an emulator trained on the GPU by the library's own forward,
backward and Adam kernels, on (theta, chi^2) pairs labelled by the plain
method's FP64 analytic likelihood; the analytic likelihood measures its error
along sampled chains."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


def test_training_reduces_emulator_error_along_chains():
    from paper_2606_04895_gb300 import Sampler
    from paper_2606_04895_gb300 import learn
    tgt = S.target(6, seed=0)
    emu, hist, (in_m, in_s, out_m, out_s) = learn.train_emulator(
        tgt, n_train=1 << 16, width=256, depth=3, epochs=12, batch=2048, lr=2e-3, precision="fp32", n_chains=256)
    assert hist["train_loss"][-1] < 0.2 * hist["train_loss"][0]
    assert hist["val_mse"][-1] < 0.1
    # chains of the plain method around the posterior
    plain = learn.analytic_sampler(tgt, n_chains=256, precision="fp32", seed=3)
    Lp = np.linalg.cholesky(tgt["laplace_cov"])
    th0 = tgt["theta_star"] + S.chains_init(256, 6, seed=5) @ Lp.T
    plain.init_chains(th0, tgt["lower"], tgt["upper"], mu=tgt["theta_star"], L=Lp)
    out = torch.empty((200, 256, 6), dtype=torch.float32, device="cuda")
    plain.step("mala", 200, eps=0.4, samples=out)
    truth = learn.analytic_sampler(tgt, n_chains=1, precision="fp64")
    err_trained = learn.dlogl_along_chains(emu, truth, out).cpu().numpy()
    # the same network before training
    e0 = S.emulator(6, width=256, depth=3, seed=5, in_m=in_m, in_s=in_s, out_m=out_m, out_s=out_s)
    raw = Sampler(6, 8, precision="fp32", likelihood="emulator")
    raw.set_emulator(e0["params"], 3, 256, in_m, in_s, out_m, out_s)
    err_raw = learn.dlogl_along_chains(raw, truth, out).cpu().numpy()
    print(f"|dlogL| along chains: trained median {np.median(err_trained):.3g}, untrained {np.median(err_raw):.3g}")
    assert np.median(err_trained) < 0.1 * np.median(err_raw)
    for s in (emu, plain, truth, raw):
        s.close()


def _reweighted_mean(x, w):
    """Self-normalised importance-weighted mean over all draws of x[t][chain][d] with weights
    w[t][chain], and its Monte Carlo standard error from the spread of the chains' weighted sums
    (chains are independent; within-chain correlation and weight variability both enter)."""
    Nc = (w[:, :, None] * x).sum(axis=0)  # [chain][d]
    Dc = w.sum(axis=0)                    # [chain]
    m = Nc.sum(axis=0) / Dc.sum()
    M = x.shape[1]
    se = np.sqrt(np.var(Nc - m * Dc[:, None], axis=0, ddof=1) / M) / Dc.mean()
    return m, se


def test_trained_emulator_chains_match_the_analytic_posterior():
    """The learned part end to end: the config-4 emulator (8-D sterile-shaped target, 2^20
    (theta, chi^2) pairs labelled by the FP64 analytic likelihood, 8-512x4-1 tanh, log output,
    Adam 1e-3 in batches of 4096, trained by the library's kernels) drives BF16 MALA, BF16 HMC
    and FP16 MALA chains (4096 chains).  Their moments, importance-reweighted by
    exp(logL_analytic - logL_emulator) (the analytic likelihood judges the emulator), agree with
    long analytic-likelihood MALA chains within 5 Monte Carlo standard errors.  Along the chains
    the FP16 chi^2 stays within 0.05 of the FP64 evaluation of the same network (BF16 within
    0.25).  What the trained network gains over the method without it: its logL error along the
    chains is far below the untrained network's, and its evaluations (with the reweighting's
    efficiency) outpace the plain analytic path."""
    from paper_2606_04895_gb300 import driver, learn
    tgt = S.target(8, seed=0)
    e, hist, _ = learn.train_emulator_log(tgt, epochs=40)
    assert hist["val_mse"][-1] < 1e-3, hist["val_mse"][-1]
    n, draws, thin = 4096, 1500, 10
    Lp = np.linalg.cholesky(tgt["laplace_cov"])
    th0 = tgt["theta_star"] + S.chains_init(n, 8, seed=5) @ Lp.T
    truth = learn.analytic_sampler(tgt, n_chains=1, precision="fp64")
    # reference: the plain method (analytic likelihood, FP32 path) sampled long
    a = learn.analytic_sampler(tgt, n_chains=n, precision="fp32", seed=3)
    a.init_chains(th0, tgt["lower"], tgt["upper"], mu=tgt["theta_star"], L=Lp)
    eps_a, _ = driver.burn_in(a, "mala", eps0=0.5, adapt_steps=400, cov_steps=1000)
    xa = torch.empty((2 * draws, n, 8), dtype=torch.float32, device="cuda")
    a.step("mala", 2 * draws, eps=eps_a, samples=xa)
    assert a.r_minus_1(xa) < 0.01
    xr = xa[::thin].double().cpu().numpy()
    m_ref = xr.mean(axis=(0, 1))
    se_ref = xr.mean(axis=0).std(axis=0, ddof=1) / np.sqrt(n)
    a.close()
    for prec, kernel, kw in [("bf16", "mala", {}), ("bf16", "hmc", {"n_leapfrog": 10}), ("fp16", "mala", {})]:
        s = learn.emulator_sampler(e, n, precision=prec, seed=7)
        s.init_chains(th0, tgt["lower"], tgt["upper"], mu=tgt["theta_star"], L=Lp)
        eps, _ = driver.burn_in(s, kernel, eps0=0.5 if kernel == "mala" else 0.2, adapt_steps=400,
                                cov_steps=1000 if kernel == "mala" else 200, **kw)
        steps = draws if kernel == "mala" else draws // 5
        x = torch.empty((steps, n, 8), dtype=torch.float32, device="cuda")
        s.step(kernel, steps, eps=eps, samples=x, **kw)
        assert s.r_minus_1(x) < 0.01
        xs = x[::thin if kernel == "mala" else 2].contiguous()
        pts = xs.reshape(-1, 8)
        dl = (truth.loglike(pts.double()).double() - s.loglike(pts).double()).cpu().numpy()
        w = np.exp(dl - np.median(dl)).reshape(xs.shape[0], n)
        m_rw, se_rw = _reweighted_mean(xs.double().cpu().numpy(), w)
        z = (m_rw - m_ref) / np.sqrt(se_rw ** 2 + se_ref ** 2)
        kish = w.sum() ** 2 / (w ** 2).sum() / w.size
        print(f"{prec} {kernel}: reweighted z {np.round(z, 2)}, |dlogL| median {np.median(np.abs(dl)):.3f}, "
              f"weight efficiency {kish:.3f}")
        assert np.all(np.abs(z) < 5.0), z
        assert kish > 0.5
        # precision claim along the chains: chi^2 against the FP64 evaluation of the same weights
        p = pts[:: max(1, len(pts) // 1500)][:1500]
        lg = s.loglike(p).double().cpu().numpy()
        r64 = O.Model(8, emulator=e).loglike(p.double().cpu().numpy(), grad=False)
        dchi2 = 2 * np.abs(lg - r64)
        print(f"{prec}: chi2 error vs FP64 along the chains max {dchi2.max():.4f} mean {dchi2.mean():.4f}")
        assert dchi2.max() <= (0.05 if prec == "fp16" else 0.25)
        s.close()
    # the same network before training, on the same points: the training is what makes it usable
    e0 = S.emulator(8, width=512, depth=4, seed=5, in_m=e["in_m"], in_s=e["in_s"], out_m=e["out_m"],
                    out_s=e["out_s"], out_log=1, out_floor=e["out_floor"])
    e0 = learn.fold_input_map(e0, *learn.input_whitening(tgt))
    raw = learn.emulator_sampler(e0, 8, precision="fp32")
    p = torch.as_tensor(xr[-1], dtype=torch.float32, device="cuda")
    err_raw = (raw.loglike(p).double() - truth.loglike(p.double()).double()).abs().cpu().numpy()
    tr = learn.emulator_sampler(e, 8, precision="fp32")
    err_tr = (tr.loglike(p).double() - truth.loglike(p.double()).double()).abs().cpu().numpy()
    print(f"|dlogL| at analytic posterior draws: trained median {np.median(err_tr):.3g}, "
          f"untrained {np.median(err_raw):.3g}")
    assert np.median(err_tr) < 1e-2 * np.median(err_raw)
    for h in (truth, raw, tr):
        h.close()


def test_trained_27d_emulator_nuts_stays_on_the_analytic_posterior():
    """Config-3 target (6 bounded + 21 nuisance dimensions, 2048-long data vector): a 27-512x4-1
    emulator trained by the library on 20 % box-uniform and 80 % Gaussian inputs at 1.5, 3 and 6
    sigma (the config-4 3-sigma mixture alone misses the 27-D typical set) drives BF16 NUTS on
    4096 chains from the Laplace start through a shortened burn-in: the draws converge (R - 1
    below 0.01), the emulator error along them stays small (median |dlogL| below 2 against the
    FP64 analytic likelihood) and no chain runs off to a spurious maximum (99th percentile below
    10)."""
    from paper_2606_04895_gb300 import driver, learn
    tgt = S.target(27, nuisance=True, seed=0)
    e, hist, _ = learn.train_emulator_log(tgt, epochs=30, gauss_frac=0.8, gauss_scale=(1.5, 3.0, 6.0))
    n = 4096
    s = learn.emulator_sampler(e, n, precision="bf16", seed=1)
    Lp = np.linalg.cholesky(tgt["laplace_cov"])
    th0 = tgt["theta_star"] + S.chains_init(n, 27, seed=5) @ Lp.T
    th0[:, :tgt["d_c"]] = np.clip(th0[:, :tgt["d_c"]], -2.99, 2.99)
    s.init_chains(th0, tgt["lower"], tgt["upper"], mu=tgt["theta_star"], L=Lp, gauss=tgt["gauss"])
    eps, _ = driver.burn_in(s, "nuts", eps0=0.3, n_iter=2, adapt_steps=200, cov_steps=300, chunk=20, target=0.8)
    x = torch.empty((300, n, 27), dtype=torch.float32, device="cuda")
    s.step("nuts", 300, eps=eps, samples=x, stats=False)
    rm1 = float(s.r_minus_1(x))
    truth = learn.analytic_sampler(tgt, n_chains=1, precision="fp64")
    dl = learn.dlogl_along_chains(s, truth, x[::30].contiguous()).cpu().numpy()
    print(f"27-D NUTS: eps {eps:.3f} R-1 {rm1:.4f} |dlogL| median {np.median(dl):.3f} p99 {np.quantile(dl, .99):.2f}")
    assert rm1 < 0.01
    assert np.median(dl) < 2.0
    assert np.quantile(dl, 0.99) < 10.0
    s.close()
    truth.close()
