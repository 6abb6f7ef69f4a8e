"""Per-step parity of the samplers against the FP64 oracle from identical
states and identical Philox streams.

Decisions must agree wherever they are clear of their threshold by the decision
margin (the oracle's trace gives log alpha - log u, and for NUTS the smallest
distance of any decision of the iteration); where they agree the new positions
must match (FP64: 1e-9; FP32, BF16 and FP16: 1e-3 absolute in x).  BF16 and FP16
runs are compared with the oracle's operand-rounding mode of the same type.

The margin of a chain is max(1e-3, B): B bounds how far the GPU's decision
quantity can sit from the oracle's, propagated to first order from the
per-evaluation discrepancies of the likelihood between the two (tau_L in log pi,
tau_g in the whitened gradient, twice their largest value over the chains' start
points, measured on the same handle before stepping; the largest value, because
a discrepancy made of whole rounding steps is heavy-tailed):
  MH, AIES (stretch / DE): B = 2 tau_L (two evaluations at the same points);
  MALA: B = 2 tau_L + tau_g (sqrt(2 eps d) + eps sqrt(d)) (the proposal terms and
        the proposal's shift by eps g);
  HMC, n leapfrogs, and NUTS, n leaves: B = 2 tau_L + eps sqrt(n d) tau_g (1 + eps n)
        (a random walk of n gradient discrepancies in the momentum, |q| ~ sqrt(d),
        and its drift into the position, |g| ~ sqrt(d)).
In FP32 / FP64 the discrepancies are rounding-level and B is far below 1e-3.  In
BF16 the hidden activations pass through tanh.approx before their BF16 rounding
(2^-11 relative error against a 2^-9 rounding step), so some of them round to the
neighbouring BF16 value of the oracle's: B is then of order 1e-2."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_common import emulator_case, make_emulator_sampler, oracle_emulator_model, whitening

pytestmark = pytest.mark.gpu

MARGIN = 1e-3
POS_TOL = {"fp64": 1e-9, "fp32": 1e-3, "bf16": 1e-3, "fp16": 1e-3}


def _setup(prec, n, d=8, width=256, depth=3, seed=11, **kw):
    e = emulator_case(d, width, depth, out_s=8.0, out_m=50.0)
    mu, L = whitening(d, 1, scale=0.4)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    theta0 = np.clip(mu + np.random.default_rng(9).normal(size=(n, d)) @ L.T, -2.9, 2.9)
    s = make_emulator_sampler(prec, e, n, mu=mu, L=L, lower=lower, upper=upper, theta0=theta0, seed=seed, **kw)
    m = oracle_emulator_model(e, mu=mu, L=L, lower=lower, upper=upper, bf16=(prec == "bf16"),
                              fp16=(prec == "fp16"))
    z0 = np.linalg.solve(L, (theta0 - mu).T).T
    s.tau = _tau(s, m, z0)
    return s, m, z0, mu, L


def _tau(s, m, z0):
    """Per-evaluation discrepancies of log pi and of its whitened gradient between the handle's
    initial state and the oracle at the same points: twice their largest value over the chains."""
    st = s.get_state()
    rl, rg = m.logpost(z0)
    ok = np.isfinite(rl) & np.isfinite(st["logp"])
    dl = st["logp"][ok] - rl[ok]
    dg = np.linalg.norm(st["grad"][ok] - rg[ok], axis=1)
    return 2.0 * np.max(np.abs(dl)), 2.0 * np.max(dg)


def _bound(s, kernel, d, eps, n_eval):
    """B of the module docstring for one chain (n_eval: leapfrogs of HMC / leaves of NUTS)."""
    tl, tg = getattr(s, "tau", (0.0, 0.0))
    if kernel == "mala":
        return 2 * tl + tg * (np.sqrt(2 * eps * d) + eps * np.sqrt(d))
    if kernel == "hmc" or kernel.startswith("nuts"):
        return 2 * tl + eps * np.sqrt(n_eval * d) * tg * (1 + eps * n_eval)
    return 2 * tl


def _check(prec, s, ref, samples, kernel, n, eps=0.0, n_leapfrog=1, margin=MARGIN, pos_tol=None):
    acc_gpu = s.counters()["accepts"]
    x_gpu = samples[-1].double().cpu().numpy()
    x_ref = ref["samples"][-1]
    d = x_ref.shape[-1]
    if kernel.startswith("nuts"):
        # every decision of a NUTS iteration (slice, Delta_max, merges, top-level moves, U-turn
        # tests) is at least the chain's margin away from its threshold on the clear chains (the
        # oracle's trace gives the smallest distance): there the tree, the leapfrog count and the
        # selected point must be the oracle's
        mc = np.maximum(margin, _bound(s, kernel, d, eps, ref["nleaf"][-1]))
        clear = ref["margin"][-1] > mc
        # (FP32 / FP64: nearly every chain; BF16: the chains clear of its larger margin)
        assert clear.mean() > 0.9 if prec in ("fp32", "fp64") else clear.sum() >= 10, (clear.mean(), clear.sum())
        same = np.all(np.abs(x_gpu - x_ref) < POS_TOL[prec], axis=1)
        assert np.all(same[clear]), np.flatnonzero(clear & ~same)
        ev = s.counters()["evals"]
        assert np.array_equal(ev[clear], ref["evals"][clear])
        return
    la, lu = ref["log_alpha"][-1], ref["log_u"][-1]
    mc = max(margin, _bound(s, kernel, d, eps, n_leapfrog))
    clear = np.abs(la - lu) > mc
    if kernel.startswith("aies"):
        # the second half of an ensemble proposes from the first half's new positions: where a
        # first-half decision inside the margin went the other way, the second half's proposals
        # differ, so those walkers are not compared
        W = 64
        acc_g, acc_r = acc_gpu.reshape(-1, 2, W // 2) > 0, ref["accept"][-1].reshape(-1, 2, W // 2) > 0
        flipped = np.any(acc_g[:, 0] != acc_r[:, 0], axis=1)
        clear = clear.reshape(-1, 2, W // 2)
        clear[flipped, 1] = False
        clear = clear.reshape(-1)
    assert clear.mean() > (0.9 if prec in ("fp32", "fp64") else 0.1), clear.mean()
    bad = np.flatnonzero(clear & ((acc_gpu > 0) != (ref["accept"][-1] > 0)))
    assert bad.size == 0, (mc, getattr(s, "tau", None), bad, (la - lu)[bad])
    tol = POS_TOL[prec] if pos_tol is None else np.asarray(pos_tol)[clear][:, None]
    assert np.all(np.abs(x_gpu[clear] - x_ref[clear]) < tol)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
@pytest.mark.parametrize("kernel,eps,extra", [("mh", 0.5, {}), ("mala", 0.4, {}), ("hmc", 0.2, {"n_leapfrog": 5}),
                                              ("nuts", 0.3, {}), ("nuts_multinomial", 0.3, {})])
def test_one_step_parity(prec, kernel, eps, extra):
    n = 300
    s, m, z0, mu, L = _setup(prec, n)
    out = torch.empty((1, n, 8), dtype=s.dtype, device="cuda")
    s.step(kernel, 1, eps=eps, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=1, seed=11, trace=True, **extra)
    _check(prec, s, ref, out, kernel, n, eps=eps, n_leapfrog=extra.get("n_leapfrog", 1))
    s.close()


@pytest.mark.parametrize("kernel", ["aies", "aies_de"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_aies_one_step_parity(prec, kernel):
    """The stretch move and the differential-evolution move (sigma_gamma = 0.1, passed as eps),
    one ensemble update of 4 ensembles of 64 walkers, and three more updates in FP64 (where the
    halves span two tiles synchronised by a cluster barrier between half-steps)."""
    n = 256  # 4 ensembles of 64 walkers
    s, m, z0, mu, L = _setup(prec, n)
    out = torch.empty((1, n, 8), dtype=s.dtype, device="cuda")
    # (FP64 emulator tiles hold 16 rows: each 32-walker half spans a cluster of two tiles)
    s.step(kernel, 1, eps=0.1, samples=out)
    ref = O.run(m, kernel, z0, eps=0.0, n_steps=1, seed=11, trace=True, aies_walkers=64, de_sigma=0.1)
    _check(prec, s, ref, out, kernel, n)
    s.close()


@pytest.mark.parametrize("kernel,eps,extra", [("mala", 0.4, {}), ("hmc", 0.25, {"n_leapfrog": 4}), ("mh", 0.5, {}),
                                              ("nuts", 0.3, {}), ("nuts_multinomial", 0.3, {})])
def test_fp64_trajectories_track_oracle(kernel, eps, extra):
    n, steps = 160, 12
    s, m, z0, mu, L = _setup("fp64", n)
    out = torch.empty((steps, n, 8), dtype=torch.float64, device="cuda")
    s.step(kernel, steps, eps=eps, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=steps, seed=11, trace=True, **extra)
    x = out.cpu().numpy()
    same = np.all(np.abs(x - ref["samples"]) < 1e-8, axis=(0, 2))
    assert same.mean() >= 0.98, same.mean()
    st = s.get_state()
    assert np.all(st["iter"] == steps)
    s.close()


def test_step_statistics_and_counters():
    n = 128
    s, m, z0, mu, L = _setup("fp32", n)
    st = s.step("hmc", 3, eps=0.2, n_leapfrog=4)
    c = s.counters()
    assert st["evals"] == n * 3 * 4 and c["evals"].sum() == n * 3 * 4
    assert st["accepts"] == c["accepts"].sum()
    assert 0.0 < st["accept_stat"] <= 1.0
    st2 = s.step("mh", 2, eps=0.3)
    assert st2["evals"] == n * 2
    s.close()


def test_checkpoint_resume_is_bit_identical():
    n = 96
    a, m, z0, mu, L = _setup("fp32", n)
    b, *_ = _setup("fp32", n)
    a.step("mala", 10, eps=0.3, stats=False)
    snap = b.get_state()
    b.step("mala", 5, eps=0.3, stats=False)
    mid = b.get_state()
    b.close()
    c, *_ = _setup("fp32", n)
    c.set_state(mid)
    c.step("mala", 5, eps=0.3, stats=False)
    sa, sc = a.get_state(), c.get_state()
    assert np.array_equal(sa["z"], sc["z"]) and np.array_equal(sa["iter"], sc["iter"])
    assert snap["iter"].max() == 0
    a.close(); c.close()


def test_samples_into_pinned_host_memory():
    """The sample record can go straight to page-locked host memory (the kernel writes it over
    the host link): bit-identical to the record in device memory from the same start, and a
    pageable host buffer is refused by the library before anything runs."""
    import ctypes as C
    from paper_2606_04895_gb300 import KERNELS
    n, k = 256, 5
    a, _, _ = _setup_gauss("bf16", n, 512)
    b, _, _ = _setup_gauss("bf16", n, 512)
    dev = torch.empty((k, n, 8), dtype=a.dtype, device="cuda")
    a.step("mala", k, eps=0.3, samples=dev, stats=False)
    host = torch.full((k, n, 8), float("nan"), dtype=b.dtype).pin_memory()
    b.step("mala", k, eps=0.3, samples=host, stats=False)
    torch.cuda.synchronize()
    assert torch.equal(host, dev.cpu())
    assert np.array_equal(a.get_state()["z"], b.get_state()["z"])
    pageable = np.zeros((k, n, 8), dtype=np.float32)
    rc = b.lib.bst_step(b.h, KERNELS["mala"], 0.3, 10, k, pageable.ctypes.data_as(C.c_void_p), None, None)
    assert rc != 0
    assert not pageable.any()
    with pytest.raises(Exception):
        b.step("mala", k, eps=0.3, samples=torch.zeros((k, n, 8), dtype=b.dtype))
    a.close(); b.close()


def test_thinning_and_sample_shape():
    from paper_2606_04895_gb300 import Sampler
    n = 64
    s, m, z0, mu, L = _setup("fp32", n, thin=3)
    out = torch.empty((4, n, 8), dtype=torch.float32, device="cuda")
    s.step("mh", 12, eps=0.3, samples=out)
    ref = O.run(m, "mh", z0, eps=0.3, n_steps=12, seed=11)
    x = out.double().cpu().numpy()
    same = np.all(np.abs(x - ref["samples"][2::3]) < 1e-3, axis=(0, 2))
    assert same.mean() > 0.9
    s.close()


def _setup_gauss(prec, n, width, d=8, seed=11, depth=3):
    """d = 8 with the last two dimensions under N(0, 1) priors (no box): exercises the prior
    terms of the register-resident BF16 chains (d <= 8)."""
    e = emulator_case(d, width, depth, out_s=8.0, out_m=50.0)
    mu, L = whitening(d, 2, scale=0.4)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    lower[6:], upper[6:] = -1e30, 1e30
    gauss = np.array([0] * 6 + [1] * 2, dtype=np.int32)
    theta0 = mu + np.random.default_rng(4).normal(size=(n, d)) @ L.T
    theta0[:, :6] = np.clip(theta0[:, :6], -2.9, 2.9)
    s = make_emulator_sampler(prec, e, n, mu=mu, L=L, lower=lower, upper=upper, theta0=theta0, gauss=gauss,
                              seed=seed)
    m = oracle_emulator_model(e, mu=mu, L=L, lower=lower, upper=upper, gauss=gauss, bf16=(prec == "bf16"),
                              fp16=(prec == "fp16"))
    z0 = np.linalg.solve(L, (theta0 - mu).T).T
    s.tau = _tau(s, m, z0)
    return s, m, z0


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("width", [256, 512])
@pytest.mark.parametrize("kernel,eps,extra", [("mh", 0.5, {}), ("mala", 0.4, {}), ("hmc", 0.2, {"n_leapfrog": 5})])
def test_bf16_register_chains_gaussian_prior_parity(width, kernel, eps, extra, prec):
    n = 300
    s, m, z0 = _setup_gauss(prec, n, width)
    out = torch.empty((1, n, 8), dtype=s.dtype, device="cuda")
    s.step(kernel, 1, eps=eps, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=1, seed=11, trace=True, **extra)
    # BF16 log alpha after five leapfrogs differs from the oracle's BF16-emulation mode (exact
    # tanh, FP64 sums) by up to a few 1e-3, so HMC decisions are compared outside 1e-2
    _check(prec, s, ref, out, kernel, n, eps=eps, n_leapfrog=extra.get("n_leapfrog", 1))
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("kernel,extra", [("mala", {}), ("hmc", {"n_leapfrog": 3}), ("mh", {})])
def test_bf16_register_chains_record_every_step(kernel, extra, prec):
    """The register-resident chains write their state, counters and samples while the next
    evaluation runs: after a launch every step's sample, the counters and the state agree
    with the oracle run step by step, and the last sample is x of the final state."""
    n, steps = 256, 6
    s, m, z0 = _setup_gauss(prec, n, 512)
    out = torch.full((steps, n, 8), float("nan"), dtype=s.dtype, device="cuda")
    s.step(kernel, steps, eps=0.3 if kernel != "hmc" else 0.15, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=0.3 if kernel != "hmc" else 0.15, n_steps=steps, seed=11, trace=True, **extra)
    x = out.double().cpu().numpy()
    assert np.isfinite(x).all()
    same = np.all(np.abs(x - ref["samples"]) < 2e-3, axis=(0, 2))
    assert same.mean() >= 0.9, same.mean()
    st = s.get_state()
    c = s.counters()
    nl = extra.get("n_leapfrog", 1)
    assert np.all(st["iter"] == steps)
    assert np.all(c["evals"] == steps * nl)
    assert np.array_equal(c["accepts"][same], ref["accepts"][same])
    mu, L = s.whitening()
    x_state = mu + st["z"] @ L.T
    assert np.max(np.abs(x_state - x[-1])) < 1e-5
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("width", [256, 512])
def test_bf16_mala_two_cta_clusters(width, prec):
    """MALA with 6000 chains (clusters of two CTAs per 128-chain tile) against the oracle."""
    n = 6000
    s, m, z0 = _setup_gauss(prec, n, width, depth=2)
    out = torch.empty((1, n, 8), dtype=s.dtype, device="cuda")
    s.step("mala", 1, eps=0.4, samples=out)
    ref = O.run(m, "mala", z0, eps=0.4, n_steps=1, seed=11, trace=True)
    _check(prec, s, ref, out, "mala", n, eps=0.4)
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_bf16_mala_headline_shape(prec):
    """The benchmark's launch configuration: 4096 chains of the 8-D target on an 8-512x4-1
    emulator (32 tiles, each on a cluster of four CTAs with the exchange through global slice
    images), one MALA step against the oracle on every chain."""
    n = 4096
    s, m, z0 = _setup_gauss(prec, n, 512, depth=4)
    # an accepted proposal differs from the oracle's by eps L (g_gpu - g_ref) at the start: the
    # position tolerance of each chain is that difference, measured, twice, plus 1e-3
    g_gpu = s.get_state()["grad"]
    _, g_ref = m.logpost(z0)
    mu, L = s.whitening()
    pos_tol = 1e-3 + 2.0 * 0.4 * np.max(np.abs((g_gpu - g_ref) @ L.T), axis=1)
    out = torch.empty((1, n, 8), dtype=s.dtype, device="cuda")
    s.step("mala", 1, eps=0.4, samples=out)
    ref = O.run(m, "mala", z0, eps=0.4, n_steps=1, seed=11, trace=True)
    _check(prec, s, ref, out, "mala", n, eps=0.4, pos_tol=pos_tol)
    print(f"{prec}: position tolerance median {np.median(pos_tol):.2e} max {pos_tol.max():.2e}")
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_bf16_mala_one_cta_per_tile_width512(prec):
    """MALA with 10,240 chains (80 tiles: one CTA per tile, the layer in two MMA halves, the
    epilogue in quarters overlapping the next layer's MMAs) against the oracle."""
    n = 10240
    s, m, z0 = _setup_gauss(prec, n, 512, depth=2)
    out = torch.empty((1, n, 8), dtype=s.dtype, device="cuda")
    s.step("mala", 1, eps=0.4, samples=out)
    ref = O.run(m, "mala", z0, eps=0.4, n_steps=1, seed=11, trace=True)
    _check(prec, s, ref, out, "mala", n, eps=0.4)
    s.close()


def _setup27(prec, n, width=256, depth=2, seed=11):
    """d = 27: six box-bounded dimensions and 21 nuisance dimensions under N(0, 1) priors, with
    a dense whitening factor (the general sampler code: chain vectors in global memory,
    FP32-first decisions)."""
    d = 27
    e = emulator_case(d, width, depth, out_s=8.0, out_m=50.0)
    mu, L = whitening(d, 3, scale=0.3)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    lower[6:], upper[6:] = -1e30, 1e30
    gauss = np.array([0] * 6 + [1] * 21, dtype=np.int32)
    theta0 = mu + np.random.default_rng(6).normal(size=(n, d)) @ L.T
    theta0[:, :6] = np.clip(theta0[:, :6], -2.9, 2.9)
    s = make_emulator_sampler(prec, e, n, mu=mu, L=L, lower=lower, upper=upper, theta0=theta0, gauss=gauss,
                              seed=seed)
    m = oracle_emulator_model(e, mu=mu, L=L, lower=lower, upper=upper, gauss=gauss, bf16=(prec == "bf16"),
                              fp16=(prec == "fp16"))
    z0 = np.linalg.solve(L, (theta0 - mu).T).T
    s.tau = _tau(s, m, z0)
    return s, m, z0


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("kernel,eps,extra", [("mh", 0.6, {}), ("mala", 0.6, {}), ("hmc", 0.5, {"n_leapfrog": 4}),
                                              ("nuts", 0.5, {}), ("nuts_multinomial", 0.5, {}),
                                              ("aies", 0.0, {"aies_walkers": 64}),
                                              ("aies_de", 0.1, {"aies_walkers": 64, "de_sigma": 0.1})])
def test_27d_one_step_parity(prec, kernel, eps, extra):
    # four AIES ensembles of 64 walkers; NUTS in BF16 / FP16 on more chains, since at d = 27 only
    # a few percent of its trees clear the margin of those precisions
    n = 1024 if (kernel.startswith("nuts") and prec in ("bf16", "fp16")) else 256
    s, m, z0 = _setup27(prec, n)
    out = torch.empty((1, n, 27), dtype=s.dtype, device="cuda")
    kw = {k: v for k, v in extra.items() if k not in ("aies_walkers", "de_sigma")}
    s.step(kernel, 1, eps=eps, samples=out, **kw)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=1, seed=11, trace=True, **extra)
    _check(prec, s, ref, out, kernel, n, eps=eps, n_leapfrog=extra.get("n_leapfrog", 1))
    s.close()


@pytest.mark.parametrize("prec", ["bf16"])
@pytest.mark.parametrize("kernel,eps", [("mala", 0.6), ("nuts", 0.5)])
def test_27d_one_cta_per_tile_parity(prec, kernel, eps):
    """The general sampler code at 10,240 chains of the 27-D target on a width-512 emulator:
    80 tiles, one CTA each, the layer in two MMA halves and the epilogue in quarters (the
    configuration the 27-D NUTS and AIES legs run at).  One step against the oracle on every
    chain."""
    n = 10240
    s, m, z0 = _setup27(prec, n, width=512, depth=2)
    out = torch.empty((1, n, 27), dtype=s.dtype, device="cuda")
    s.step(kernel, 1, eps=eps, samples=out)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=1, seed=11, trace=True)
    _check(prec, s, ref, out, kernel, n, eps=eps)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("kernel,eps,extra", [("mala", 0.6, {}), ("nuts", 0.5, {}), ("hmc", 0.4, {"n_leapfrog": 3}),
                                              ("aies", 0.0, {})])
def test_27d_trajectories_and_counters(prec, kernel, eps, extra):
    """Five iterations of the general code at d = 27: samples, counters and the final state
    against the oracle run step by step."""
    n, steps = 256, 5
    s, m, z0 = _setup27(prec, n)
    out = torch.full((steps, n, 27), float("nan"), dtype=s.dtype, device="cuda")
    s.step(kernel, steps, eps=eps, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=steps, seed=11, trace=True, **extra)
    x = out.double().cpu().numpy()
    assert np.isfinite(x).all()
    same = np.all(np.abs(x - ref["samples"]) < 2e-3, axis=(0, 2))
    assert same.mean() >= 0.9, same.mean()
    st = s.get_state()
    c = s.counters()
    assert np.all(st["iter"] == steps)
    assert np.array_equal(c["accepts"][same], ref["accepts"][same])
    # a U-turn test that flips under BF16 rounding adds a doubling whose candidate need not be
    # taken: the same samples can come with a different leapfrog count
    assert np.mean(c["evals"][same] == ref["evals"][same]) >= 0.95
    mu, L = s.whitening()
    assert np.max(np.abs(mu + st["z"] @ L.T - x[-1])) < 1e-4
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("kernel,eps,extra", [("mala", 0.6, {}), ("nuts", 0.5, {}), ("mh", 0.6, {})])
def test_27d_ragged_chain_count(prec, kernel, eps, extra):
    """200 chains: the last block of 32 chains of the chain-blocked buffers and the last
    128-chain tile are partly empty."""
    n = 200
    s, m, z0 = _setup27(prec, n)
    out = torch.empty((2, n, 27), dtype=s.dtype, device="cuda")
    s.step(kernel, 2, eps=eps, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=2, seed=11, trace=True, **extra)
    x = out.double().cpu().numpy()
    same = np.all(np.abs(x - ref["samples"]) < 2e-3, axis=(0, 2))
    assert same.mean() >= 0.9, same.mean()
    assert np.all(s.get_state()["iter"] == 2)
    s.close()


# ---------------------------------------------------------------- smooth bounds penalty (Sec. 3.1)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("kernel,eps,extra", [("mh", 0.5, {}), ("mala", 0.4, {}), ("hmc", 0.2, {"n_leapfrog": 5}),
                                              ("nuts", 0.3, {})])
def test_bounds_penalty_one_step_parity(prec, kernel, eps, extra):
    """Bounds inside the chains' spread with smooth penalties (some chains start outside): the
    chains' log pi and gradient after bst_set_bounds_penalty, and one step of every sampler,
    against the oracle with the same penalty widths."""
    n, d = 300, 8
    e = emulator_case(d, 256, 3, out_s=8.0, out_m=50.0)
    mu, L = whitening(d, 1, scale=0.4)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    upper[0], lower[1], upper[5] = mu[0], mu[1] - 0.1, mu[5] + 0.2
    pen = np.array([0.2, 0.05, 0.0, 0.0, 0.0, 0.5, 0.0, 0.0])
    theta0 = mu + np.random.default_rng(9).normal(size=(n, d)) @ L.T
    theta0[:, 2:5] = np.clip(theta0[:, 2:5], -2.9, 2.9)
    theta0[:, 6:] = np.clip(theta0[:, 6:], -2.9, 2.9)
    s = make_emulator_sampler(prec, e, n, mu=mu, L=L, lower=lower, upper=upper, theta0=theta0, seed=11)
    s.set_bounds_penalty(pen)
    m = O.Model(d, emulator=e, lower=lower, upper=upper, mu=mu, L=L, bf16=(prec == "bf16"), pen_w=pen)
    z0 = np.linalg.solve(L, (theta0 - mu).T).T
    st = s.get_state()
    rl, rg = m.logpost(z0)
    assert np.all(np.isfinite(rl)) and np.isfinite(st["logp"]).all()
    assert (theta0[:, 0] > upper[0]).sum() > 50  # many chains start outside a smooth bound
    tl, tg = {"fp64": (1e-10, 1e-9), "fp32": (1e-5, 1e-4), "bf16": (2e-3, 2e-2)}[prec]
    assert np.max(np.abs(st["logp"] - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    from gpu_common import rel_err
    assert rel_err(st["grad"], rg) < tg
    out = torch.empty((1, n, d), dtype=s.dtype, device="cuda")
    s.tau = _tau(s, m, z0)
    s.step(kernel, 1, eps=eps, samples=out, **extra)
    ref = O.run(m, kernel, z0, eps=eps, n_steps=1, seed=11, trace=True, **extra)
    _check(prec, s, ref, out, kernel, n, eps=eps, n_leapfrog=extra.get("n_leapfrog", 1))
    s.close()
