"""GPU parity of loglike / grad_loglike and of the initial log pi against the FP64 oracle.

Tolerances: FP32 logL 1e-5 relative and gradient 1e-4 relative (of the largest
component); FP64 1e-10; BF16 and FP16 (tensor-core operands) against the oracle's
operand-rounding mode of the same type (same rounding points; FP32 vs FP64
accumulation and the tanh approximation can flip an operand rounding now and
then): BF16 2e-3 / 2e-2, FP16 3e-4 / 3e-3.  The precision claim against the FP64
evaluation of the same network (test_chi2_error_against_fp64): FP16 operands stay
within 0.05 in chi^2, the accuracy target of the path; BF16 operands (8 significant bits)
do not at the tested output scale and are held to their own arithmetic bound."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_common import emulator_case, rel_err, whitening

pytestmark = pytest.mark.gpu


def _sampler(prec, e, lik="emulator", n=8, t=None):
    from paper_2606_04895_gb300 import Sampler
    d = e["d"] if lik == "emulator" else t["d"]
    s = Sampler(d, n, precision=prec, likelihood=lik, seed=1)
    if lik == "emulator":
        s.set_emulator(e["params"], e["depth"], e["width"], e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    else:
        s.set_analytic(t["A"], t["B"], t["c"], t["data"], t["sigma"], d_c=t["d_c"], N=t["N"], linear=t["linear"])
    return s


SHAPES = [(8, 256, 1), (8, 256, 3), (6, 512, 4), (27, 512, 2)]
TOL = {"fp64": (1e-10, 1e-9), "fp32": (1e-5, 1e-4), "bf16": (2e-3, 2e-2), "fp16": (3e-4, 3e-3)}


def _ref(prec, d, e, **kw):
    """The oracle model for a precision: the operand-rounding mode for the tensor-core paths."""
    return O.Model(d, emulator=e, bf16=(prec == "bf16"), fp16=(prec == "fp16"), **kw)


@pytest.mark.parametrize("d,width,depth", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_emulator_loglike_parity(prec, d, width, depth):
    if prec == "fp64" and width > 512:
        pytest.skip("fp64 width <= 512")
    e = emulator_case(d, width, depth, out_s=20.0, out_m=100.0)
    s = _sampler(prec, e)
    m = 300  # several tiles of 16 / 32 / 128 rows plus a ragged tail
    x = np.random.default_rng(2).uniform(-3, 3, (m, d))
    ll, g = s.grad_loglike(x)
    ll0 = s.loglike(x)
    ll, g, ll0 = ll.double().cpu().numpy(), g.double().cpu().numpy(), ll0.double().cpu().numpy()
    ref = _ref(prec, d, e)
    rl, rg = ref.loglike(x)
    assert np.array_equal(ll, ll0) or rel_err(ll0, rl) < 1e-5
    tl, tg = TOL[prec]
    if prec == "fp64":
        assert rel_err(ll, rl) < tl and rel_err(g, rg) < tg
    else:
        assert np.max(np.abs(ll - rl) / np.maximum(np.abs(rl), 1.0)) < tl, np.max(np.abs(ll - rl))
        assert rel_err(g, rg) < tg
    s.close()


@pytest.mark.parametrize("prec,bound", [("fp16", 0.05), ("bf16", 0.25)])
def test_chi2_error_against_fp64(prec, bound):
    """Precision claim of the tensor-core operands: chi^2 of the emulator against the FP64 oracle
    evaluation of the same weights, element by element, at the 8-512x4-1 shape, output scale
    out_s = 20, 4000 points uniform in the box (several tiles and a ragged tail).  FP16: within
    0.05.  BF16 (2^-9 relative rounding of every weight and hidden activation, about 10x the
    FP16 error) is held to 0.25."""
    d, width, depth = 8, 512, 4
    e = emulator_case(d, width, depth, out_s=20.0, out_m=100.0)
    s = _sampler(prec, e)
    x = np.random.default_rng(12).uniform(-3, 3, (4000, d))
    ll = s.loglike(x).double().cpu().numpy()
    r64 = O.Model(d, emulator=e).loglike(x, grad=False)
    dchi2 = 2 * np.abs(ll - r64)
    print(f"{prec} |dchi2| vs FP64: max {dchi2.max():.4f} mean {dchi2.mean():.4f}")
    assert dchi2.max() <= bound
    s.close()


@pytest.mark.parametrize("d,width,depth", [(8, 512, 4), (27, 512, 2), (6, 256, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_emulator_log_output_parity(prec, d, width, depth):
    """Log output chi2 = floor + exp(out_s out + out_m): logL and gradient against the oracle
    (the BF16 path against the oracle's BF16 rounding mode), for loglike / grad_loglike and for
    the register-resident and general chains' initial log pi and gradient."""
    e = emulator_case(d, width, depth, out_s=1.2, out_m=2.5)
    e = dict(e, out_log=1, out_floor=200.0)
    from paper_2606_04895_gb300 import Sampler
    s = Sampler(d, 300, precision=prec, likelihood="emulator", seed=1)
    s.set_emulator(e["params"], depth, width, e["in_m"], e["in_s"], e["out_m"], e["out_s"], out_log=1,
                   out_floor=e["out_floor"])
    x = np.random.default_rng(4).uniform(-3, 3, (300, d))
    ll, g = s.grad_loglike(x)
    ll0 = s.loglike(x)
    ll, g, ll0 = ll.double().cpu().numpy(), g.double().cpu().numpy(), ll0.double().cpu().numpy()
    rl, rg = _ref(prec, d, e).loglike(x)
    tl, tg = TOL[prec]
    for v in (ll, ll0):
        assert np.max(np.abs(v - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    assert rel_err(g, rg) < tg
    # chains' initial log pi and gradient (whitened) through the step kernels' refresh
    mu, L = whitening(d, seed=2)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    z0 = np.random.default_rng(5).normal(size=(300, d)) * 0.8
    th0 = mu + z0 @ L.T
    s.init_chains(th0, lower, upper, mu=mu, L=L)
    st = s.get_state()
    m = _ref(prec, d, e, lower=lower, upper=upper, mu=mu, L=L)
    lp_ref, g_ref = m.logpost(np.linalg.solve(L, (th0 - mu).T).T)
    ok = np.isfinite(lp_ref)
    assert np.max(np.abs(st["logp"][ok] - lp_ref[ok]) / np.maximum(np.abs(lp_ref[ok]), 1.0)) < tl
    assert rel_err(st["grad"][ok], g_ref[ok]) < tg
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("depth", [7, 8])
def test_bf16_deep_width512(depth, prec):
    """Depth 7 keeps the stored activations of a 4-CTA cluster in tensor memory; depth 8 no
    longer fits there and runs on a smaller cluster with global scratch."""
    e = emulator_case(8, 512, depth, out_s=20.0, out_m=100.0)
    s = _sampler(prec, e)
    x = np.random.default_rng(3).uniform(-3, 3, (300, 8))
    ll, g = s.grad_loglike(x)
    rl, rg = _ref(prec, 8, e).loglike(x)
    ll, g = ll.double().cpu().numpy(), g.double().cpu().numpy()
    tl, tg = TOL[prec]
    assert np.max(np.abs(ll - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    assert rel_err(g, rg) < tg
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_loglike_edge_sizes(prec):
    e = emulator_case(8, 256, 2)
    s = _sampler(prec, e)
    ref = _ref(prec, 8, e)
    for m in (0, 1, 129):
        x = np.random.default_rng(m).uniform(-3, 3, (m, 8))
        ll, g = s.grad_loglike(torch.as_tensor(x).reshape(m, 8))
        assert ll.shape == (m,) and g.shape == (m, 8)
        if m:
            rl, rg = ref.loglike(x)
            assert np.max(np.abs(ll.double().cpu().numpy() - rl)) < 1e-2 * max(1, np.abs(rl).max())
    s.close()


TARGETS = {"lcdm6": dict(d=6), "sterile8": dict(d=8), "nuis27": dict(d=27, nuisance=True),
           "linear6": dict(d=6, linear=True)}


@pytest.mark.parametrize("name", list(TARGETS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_analytic_loglike_parity(prec, name):
    t = S.target(seed=0, **TARGETS[name])
    s = _sampler(prec, None, "analytic", t=t)
    m = 257
    x = t["theta_star"] + 0.05 * np.random.default_rng(1).normal(size=(m, t["d"]))
    ll, g = s.grad_loglike(x)
    ll, g = ll.double().cpu().numpy(), g.double().cpu().numpy()
    ref = O.Model(t["d"], lik="analytic", analytic=t)
    rl, rg = ref.loglike(x)
    tol_l, tol_g = (1e-11, 1e-9) if prec == "fp64" else (1e-5, 1e-4)
    assert np.max(np.abs(ll - rl) / np.maximum(np.abs(rl), 1.0)) < tol_l
    assert rel_err(g, rg) < tol_g
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_init_chains_log_pi_and_gradient(prec):
    d = 8
    e = emulator_case(d, 256, 3)
    mu, L = whitening(d, 3)
    lower, upper = np.full(d, -3.0), np.full(d, 3.0)
    gauss = np.array([0] * 6 + [1] * 2, dtype=np.int32)
    n = 200
    theta0 = mu + np.random.default_rng(4).normal(size=(n, d)) @ L.T
    theta0[0, 0] = 3.5  # one start outside the box: log pi = -inf
    from gpu_common import make_emulator_sampler
    s = make_emulator_sampler(prec, e, n, mu=mu, L=L, lower=lower, upper=upper, theta0=theta0, gauss=gauss)
    st = s.get_state()
    ref = _ref(prec, d, e, lower=lower, upper=upper, gauss=gauss, mu=mu, L=L)
    z0 = np.linalg.solve(L, (theta0 - mu).T).T
    assert np.allclose(st["z"], z0, rtol=0, atol={"fp64": 1e-12}.get(prec, 1e-5))
    rl, rg = ref.logpost(z0)
    assert st["logp"][0] == -np.inf and rl[0] == -np.inf
    fin = np.isfinite(rl)
    tol, tolg = TOL[prec]
    assert np.max(np.abs(st["logp"][fin] - rl[fin]) / np.maximum(np.abs(rl[fin]), 1)) < tol
    assert rel_err(st["grad"], rg) < tolg
    assert np.all(st["iter"] == 0)
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_bf16_one_cta_per_tile_width512(prec):
    """10,240 points are 80 tiles of 128: more than half the SMs' worth, so each tile runs on one
    CTA with the layer in two 256-column MMA halves and the epilogue in quarters, the next
    layer's MMAs starting on the finished quarters (8-512x4-1).  Every fifth row against the
    oracle (sampled outputs at a size the path runs at)."""
    e = emulator_case(8, 512, 4, out_s=20.0, out_m=100.0)
    s = _sampler(prec, e)
    x = np.random.default_rng(21).uniform(-3, 3, (10240, 8))
    ll, g = s.grad_loglike(x)
    sub = np.arange(0, 10240, 5)
    rl, rg = _ref(prec, 8, e).loglike(x[sub])
    ll, g = ll.double().cpu().numpy()[sub], g.double().cpu().numpy()[sub]
    tl, tg = TOL[prec]
    assert np.max(np.abs(ll - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    assert rel_err(g, rg) < tg
    # forward only (loglike) takes the same path
    lf = s.loglike(x).double().cpu().numpy()[sub]
    assert np.max(np.abs(lf - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    s.close()


def test_bf16_gradient_at_262144_rows():
    """The largest chain count of the throughput sweep: 262,144 rows of 8-512x4-1 (2048 tiles,
    one CTA each, in waves over the SMs), every 128th row against the oracle."""
    e = emulator_case(8, 512, 4, out_s=20.0, out_m=100.0)
    s = _sampler("bf16", e)
    n = 262144
    x = np.random.default_rng(23).uniform(-3, 3, (n, 8))
    ll, g = s.grad_loglike(x)
    sub = np.arange(0, n, 128)
    rl, rg = _ref("bf16", 8, e).loglike(x[sub])
    ll, g = ll.double().cpu().numpy()[sub], g.double().cpu().numpy()[sub]
    tl, tg = TOL["bf16"]
    assert np.max(np.abs(ll - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    assert rel_err(g, rg) < tg
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("width", [256, 512])
def test_bf16_two_cta_clusters(width, prec):
    """6000 points are 47 tiles of 128: the BF16 engine splits each layer over clusters of two
    CTAs (per-warp shared->shared slice exchange; width 256 keeps the stored activations in
    tensor memory, width 512 in global scratch)."""
    e = emulator_case(8, width, 2, out_s=20.0, out_m=100.0)
    s = _sampler(prec, e)
    x = np.random.default_rng(5).uniform(-3, 3, (6000, 8))
    ll, g = s.grad_loglike(x)
    rl, rg = _ref(prec, 8, e).loglike(x)
    ll, g = ll.double().cpu().numpy(), g.double().cpu().numpy()
    tl, tg = TOL[prec]
    assert np.max(np.abs(ll - rl) / np.maximum(np.abs(rl), 1.0)) < tl
    assert rel_err(g, rg) < tg
    s.close()
