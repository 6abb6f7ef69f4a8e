"""Pins for the oracle's samplers (paper Sec. 2): closed-form posterior moments
of the linear theory map (every kernel, including the multinomial NUTS variant and the
differential-evolution move), leapfrog reversibility / volume preservation and the
O(eps^2) energy error of HMC, reversibility of MH on a two-state coarse
graining, the stretch-factor law of AIES (Eq. (2.15) against g(z) of
Eq. (2.14)) and its affine invariance."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
import synthetic as S


def _linear_problem(d=6, n_data=64, seed=0):
    t = S.target(d, linear=True, seed=seed, n_data=n_data)
    J = t["A"] @ t["B"]
    y = t["data"] - t["A"] @ t["c"]
    P = J.T @ J / t["sigma"] ** 2
    cov = np.linalg.inv(P)
    mean = cov @ (J.T @ y) / t["sigma"] ** 2
    return t, mean, cov


def _model(t, mu, L, **kw):
    return O.Model(t["d"], lik="analytic", analytic=t, lower=t["lower"], upper=t["upper"],
                   gauss=t["gauss"], mu=mu, L=L, **kw)


def _check_moments(samples, mean, cov, nsig=5.0):
    """samples[n_draws][n_chains][d]; MCSE from the spread of independent chains."""
    n, M, d = samples.shape
    cm = samples.mean(axis=0)                          # per-chain means [M][d]
    m_hat = cm.mean(axis=0)
    se_m = cm.std(axis=0, ddof=1) / np.sqrt(M)
    assert np.all(np.abs(m_hat - mean) < nsig * se_m + 1e-12), (m_hat - mean) / se_m
    dev = samples - mean
    cc = np.einsum("tca,tcb->cab", dev, dev) / n      # per-chain second moments about truth
    c_hat = cc.mean(axis=0)
    se_c = cc.std(axis=0, ddof=1) / np.sqrt(M)
    z = (c_hat - cov) / se_c
    assert np.all(np.abs(z) < nsig), z


@pytest.mark.parametrize("kernel,eps,steps,extra", [
    ("mh", 0.3, 3000, {}),
    ("mala", 0.3, 3000, {}),
    ("hmc", 0.25, 1000, {"n_leapfrog": 10}),
    ("nuts", 0.35, 1000, {"max_depth": 8}),
    # large step: many leaves fall outside the slice, so the in-subtree and
    # top-level selection probabilities matter
    ("nuts", 1.3, 3000, {"max_depth": 8}),
    ("hmc", 0.9, 1500, {"n_leapfrog": 3}),
    # multinomial NUTS: trajectory points weighted by exp(-H), at a small and a large step
    ("nuts_multinomial", 0.35, 1000, {"max_depth": 8}),
    ("nuts_multinomial", 1.3, 3000, {"max_depth": 8}),
])
def test_closed_form_posterior(kernel, eps, steps, extra):
    t, mean, cov = _linear_problem()
    Lp = np.linalg.cholesky(cov)
    # deliberately imperfect whitening: the sampler must still be exact
    mu = mean + 0.3 * np.sqrt(np.diag(cov))
    L = 1.2 * Lp
    m = _model(t, mu, L)
    z0 = np.linalg.solve(L, (mean + S.chains_init(64, 6, seed=7) @ Lp.T - mu).T).T
    r = O.run(m, kernel, z0, eps=eps, n_steps=steps, seed=42, **extra)
    keep = r["samples"][steps // 5:]
    _check_moments(keep, mean, cov)
    acc = r["accepts"].sum() / (64 * steps)
    assert 0.05 < acc <= 1.0


def test_aies_closed_form_posterior():
    t, mean, cov = _linear_problem()
    Lp = np.linalg.cholesky(cov)
    m = _model(t, np.zeros(6), np.eye(6))
    n_ens = 32
    x0 = mean + S.chains_init(n_ens * 64, 6, seed=8) @ Lp.T
    steps = 800
    r = O.run(m, "aies", x0, eps=0.0, n_steps=steps, seed=3, aies_walkers=64)
    keep = r["samples"][steps // 4:]
    # walkers of one ensemble are correlated: use ensembles as the independent units
    ens = keep.reshape(keep.shape[0], n_ens, 64, 6).transpose(0, 2, 1, 3).reshape(-1, n_ens, 6)
    _check_moments(ens, mean, cov)


def test_hmc_energy_error_is_second_order():
    t, mean, cov = _linear_problem()
    m = _model(t, mean, np.linalg.cholesky(cov))
    z0 = S.chains_init(256, 6, seed=1)
    rms = []
    epss = [0.2, 0.1, 0.05]
    for eps in epss:
        Lf = int(round(1.0 / eps))
        r = O.run(m, "hmc", z0, eps=eps, n_leapfrog=Lf, n_steps=1, seed=5, trace=True)
        rms.append(np.sqrt(np.mean(r["log_alpha"] ** 2)))
    slope = np.polyfit(np.log(epss), np.log(rms), 1)[0]
    assert abs(slope - 2.0) < 0.1, slope


def test_leapfrog_reversible_and_volume_preserving():
    t = S.target(2, seed=4, n_data=32)
    m = _model(t, np.zeros(2), np.eye(2) * 0.05)
    z = np.array([0.3, -0.2]) + np.linalg.solve(np.eye(2) * 0.05, t["theta_star"])
    _, g = m.logpost(z[None])
    q = np.array([0.7, -1.1])
    z1, q1, g1, _ = O.leapfrog(m, z, q, g[0], 0.05, 15)
    z2, q2, _, _ = O.leapfrog(m, z1, -q1, g1, 0.05, 15)
    assert np.allclose(z2, z, atol=1e-10) and np.allclose(-q2, q, atol=1e-10)

    def phi(v):
        zz, qq = v[:2], v[2:]
        _, gg = m.logpost(zz[None])
        a, b, _, _ = O.leapfrog(m, zz, qq, gg[0], 0.05, 15)
        return np.concatenate([a, b])

    v0 = np.concatenate([z, q])
    Jm = np.zeros((4, 4))
    h = 1e-6
    for i in range(4):
        e = np.zeros(4); e[i] = h
        Jm[:, i] = (phi(v0 + e) - phi(v0 - e)) / (2 * h)
    assert abs(np.linalg.det(Jm) - 1.0) < 1e-5


def test_mh_detailed_balance_coarse_grained():
    """Coarse-grain a 1-D MH chain into three intervals.  Detailed balance makes
    the i->j and j->i transition counts equal in expectation for every pair
    (a non-reversible kernel could circulate A->B->C->A); the occupancy of an
    interval of the linear (Gaussian) target is its normal probability."""
    t, mean, cov = _linear_problem(d=1, n_data=16, seed=2)
    sd = np.sqrt(cov[0, 0])
    m = _model(t, mean, np.array([[sd]]))
    z0 = S.chains_init(256, 1, seed=4)
    r = O.run(m, "mh", z0, eps=2.0, n_steps=4000, seed=9)
    x = (r["samples"][:, :, 0] - mean[0]) / sd
    cut = np.array([-0.3, 0.8])
    st = np.digitize(x, cut)
    for i in range(3):
        for j in range(i + 1, 3):
            nij = np.sum((st[:-1] == i) & (st[1:] == j))
            nji = np.sum((st[:-1] == j) & (st[1:] == i))
            assert nij > 1000 and abs(nij - nji) < 5 * np.sqrt(nij + nji), (i, j, nij, nji)
    occ = (st == 1).mean(axis=0)
    p_b = stats.norm.cdf(0.8) - stats.norm.cdf(-0.3)
    assert abs(occ.mean() - p_b) < 5 * occ.std(ddof=1) / np.sqrt(occ.size)


def test_aies_stretch_factor_law():
    """d = 1, flat target: every stretch is accepted and, with all partners at 0
    and the moving walkers at 1, the new position is the stretch factor Z."""
    d, a = 1, 2.0
    e = S.emulator(d, width=8, depth=1, seed=0)
    W, b, wo, bo = S.unpack_emulator(e)
    flat = dict(e, params=S.pack_emulator([np.zeros_like(W[0])], b, np.zeros_like(wo), 0.0))
    m = O.Model(d, emulator=flat, lower=[-100.0], upper=[100.0])
    n_ens, W_ = 200, 64
    z0 = np.zeros((n_ens * W_, 1))
    for e_ in range(n_ens):
        z0[e_ * W_: e_ * W_ + 32] = 1.0
    r = O.run(m, "aies", z0, eps=0.0, n_steps=1, seed=21, aies_walkers=W_, aies_a=a)
    Z = np.concatenate([r["samples"][0, e_ * W_: e_ * W_ + 32, 0] for e_ in range(n_ens)])
    assert Z.min() >= 1 / a and Z.max() <= a
    F = lambda z: (np.sqrt(z) - 1 / np.sqrt(a)) / (np.sqrt(a) - 1 / np.sqrt(a))
    assert stats.kstest(Z, F).pvalue > 1e-4
    assert r["accepts"][: 32].sum() == 32


def test_aies_affine_invariance():
    t, mean, cov = _linear_problem()
    rng = np.random.default_rng(3)
    Mx = np.tril(rng.normal(size=(6, 6))) * 0.3 + np.eye(6)
    bvec = rng.normal(size=6) * 0.1
    m1 = _model(t, np.zeros(6), np.eye(6))
    m2 = _model(t, bvec, Mx)
    x0 = mean + S.chains_init(128, 6, seed=2) @ np.linalg.cholesky(cov).T
    z0 = np.linalg.solve(Mx, (x0 - bvec).T).T
    r1 = O.run(m1, "aies", x0, eps=0.0, n_steps=50, seed=13)
    r2 = O.run(m2, "aies", z0, eps=0.0, n_steps=50, seed=13)
    assert np.array_equal(r1["accepts"], r2["accepts"])
    assert np.allclose(r1["samples"], r2["samples"], rtol=1e-9, atol=1e-9)


def test_nuts_tree_bookkeeping():
    t, mean, cov = _linear_problem()
    m = _model(t, mean, np.linalg.cholesky(cov))
    z0 = S.chains_init(64, 6, seed=1)
    r = O.run(m, "nuts", z0, eps=0.3, n_steps=20, seed=3, max_depth=8, trace=True)
    depth, nleaf = r["depth"], r["nleaf"]
    assert np.all((depth >= 1) & (depth <= 8))
    # leapfrogs per iteration lie between 2^(j-1) (first doubling of the last depth)
    # and 2^j - 1 (all doublings complete)
    assert np.all(nleaf <= 2 ** depth - 1) and np.all(nleaf >= 2 ** (depth - 1))
    assert r["evals"].sum() == nleaf.sum()
    # max_depth caps the tree
    r1 = O.run(m, "nuts", z0, eps=0.01, n_steps=3, seed=3, max_depth=3, trace=True)
    assert np.all(r1["depth"] == 3) and np.all(r1["nleaf"] == 7)


def test_mala_proposal_reduces_to_gaussian_kernel():
    """On the whitened exact Gaussian N(0, I) (grad = -z) the MALA proposal mean is
    (1 - eps) z and its log-acceptance depends only on the two points; with eps -> 0
    every proposal is accepted."""
    t, mean, cov = _linear_problem()
    m = _model(t, mean, np.linalg.cholesky(cov))
    z0 = S.chains_init(256, 6, seed=6)
    r = O.run(m, "mala", z0, eps=1e-6, n_steps=3, seed=1, trace=True)
    assert np.all(r["accept"] == 1)
    assert np.all(np.abs(r["log_alpha"]) < 1e-3)


# ---- differential-evolution move (Sec. 2.3, after Eq. (2.15)) ----

def test_aies_de_closed_form_posterior():
    t, mean, cov = _linear_problem()
    Lp = np.linalg.cholesky(cov)
    m = _model(t, np.zeros(6), np.eye(6))
    n_ens = 32
    x0 = mean + S.chains_init(n_ens * 64, 6, seed=9) @ Lp.T
    steps = 800
    r = O.run(m, "aies_de", x0, eps=0.0, n_steps=steps, seed=4, aies_walkers=64, de_sigma=0.1)
    keep = r["samples"][steps // 4:]
    ens = keep.reshape(keep.shape[0], n_ens, 64, 6).transpose(0, 2, 1, 3).reshape(-1, n_ens, 6)
    _check_moments(ens, mean, cov)
    assert 0.1 < r["accepts"].sum() / (n_ens * 64 * steps) < 0.9


def _flat_1d():
    e = S.emulator(1, width=8, depth=1, seed=0)
    W, b, wo, bo = S.unpack_emulator(e)
    flat = dict(e, params=S.pack_emulator([np.zeros_like(W[0])], b, np.zeros_like(wo), 0.0))
    return O.Model(1, emulator=flat, lower=[-1000.0], upper=[1000.0])


def test_aies_de_partner_law():
    """d = 1, flat target, de_sigma = 0: the moving half at 1, the other half at 0..31.  Every
    move is accepted and y - 1 = gamma0 (p_j - p_k), gamma0 = 2.38 / sqrt(2): the difference
    j - k is never 0 (two distinct partners) and takes delta with probability
    (32 - |delta|) / (32 * 31) (an ordered pair of distinct walkers, uniform)."""
    m = _flat_1d()
    n_ens, W_ = 400, 64
    z0 = np.zeros((n_ens * W_, 1))
    for e_ in range(n_ens):
        z0[e_ * W_: e_ * W_ + 32, 0] = 1.0
        z0[e_ * W_ + 32: (e_ + 1) * W_, 0] = np.arange(32)
    r = O.run(m, "aies_de", z0, eps=0.0, n_steps=1, seed=22, aies_walkers=W_, de_sigma=0.0)
    y = np.concatenate([r["samples"][0, e_ * W_: e_ * W_ + 32, 0] for e_ in range(n_ens)])
    D = (y - 1.0) / (2.38 / np.sqrt(2.0))
    Di = np.rint(D)
    assert np.allclose(D, Di, atol=1e-9)
    assert np.all(Di != 0) and np.abs(Di).max() <= 31
    deltas = np.arange(-31, 32)
    deltas = deltas[deltas != 0]
    expect = (32 - np.abs(deltas)) / (32 * 31) * D.size
    obs = np.array([(Di == dl).sum() for dl in deltas])
    assert stats.chisquare(obs, expect).pvalue > 1e-4


def test_aies_de_gamma_law():
    """d = 1, flat target, de_sigma = 0.3: the other half has 16 walkers at 0 and 16 at 1, so
    (y - 1) / gamma0 is exactly 0 with probability 2 * 16 * 15 / (32 * 31) and otherwise
    +-(1 + eta), eta ~ N(0, 0.3^2)."""
    m = _flat_1d()
    n_ens, W_, sig = 600, 64, 0.3
    z0 = np.zeros((n_ens * W_, 1))
    for e_ in range(n_ens):
        z0[e_ * W_: e_ * W_ + 32, 0] = 1.0
        z0[e_ * W_ + 48: (e_ + 1) * W_, 0] = 1.0
    r = O.run(m, "aies_de", z0, eps=0.0, n_steps=1, seed=23, aies_walkers=W_, de_sigma=sig)
    y = np.concatenate([r["samples"][0, e_ * W_: e_ * W_ + 32, 0] for e_ in range(n_ens)])
    v = (y - 1.0) / (2.38 / np.sqrt(2.0))
    zero = v == 0.0
    p0 = 2 * 16 * 15 / (32 * 31)
    assert abs(zero.mean() - p0) < 5 * np.sqrt(p0 * (1 - p0) / v.size)
    mix = lambda u: 0.5 * stats.norm.cdf(u, 1.0, sig) + 0.5 * stats.norm.cdf(u, -1.0, sig)
    assert stats.kstest(v[~zero], mix).pvalue > 1e-4


def test_aies_de_affine_invariance_and_argument_checks():
    t, mean, cov = _linear_problem()
    rng = np.random.default_rng(5)
    Mx = np.tril(rng.normal(size=(6, 6))) * 0.3 + np.eye(6)
    bvec = rng.normal(size=6) * 0.1
    m1 = _model(t, np.zeros(6), np.eye(6))
    m2 = _model(t, bvec, Mx)
    x0 = mean + S.chains_init(128, 6, seed=3) @ np.linalg.cholesky(cov).T
    z0 = np.linalg.solve(Mx, (x0 - bvec).T).T
    r1 = O.run(m1, "aies_de", x0, eps=0.0, n_steps=50, seed=14)
    r2 = O.run(m2, "aies_de", z0, eps=0.0, n_steps=50, seed=14)
    assert np.array_equal(r1["accepts"], r2["accepts"])
    assert np.allclose(r1["samples"], r2["samples"], rtol=1e-9, atol=1e-9)
    with pytest.raises(ValueError):
        O.run(m1, "aies_de", x0[:2], eps=0.0, n_steps=1, seed=1, aies_walkers=2)  # needs 2 partners
    with pytest.raises(ValueError):
        O.run(m1, "aies_de", x0, eps=0.0, n_steps=1, seed=1, de_sigma=-1.0)


# ---------------------------------------------------------------- smooth bounds penalty (Sec. 3.1)
def _penalised_marginal_mean(mu_k, sd_k, w):
    """Marginal mean of x_k under N(mu, Sigma) times exp(-((x_k - mu_k)_+ / w)^2 / 2) (the upper
    bound of dim k at its posterior mean, penalty width w): the x_k marginal is a left half-normal
    of scale sd_k and a right half-normal of scale s' = sd_k w / sqrt(sd_k^2 + w^2), with masses
    in the ratio sd_k : s', so its mean is mu_k + sqrt(2 / pi) (s' - sd_k)."""
    sp = sd_k * w / np.sqrt(sd_k ** 2 + w ** 2)
    return mu_k + np.sqrt(2.0 / np.pi) * (sp - sd_k)


def test_bounds_penalty_is_zero_inside_and_continuous_at_the_bound():
    t, mean, cov = _linear_problem()
    L = np.linalg.cholesky(cov)
    upper = t["upper"].copy()
    upper[0] = mean[0]
    w = np.full(6, 0.05)
    hard = O.Model(6, lik="analytic", analytic=t, lower=t["lower"], upper=upper, mu=mean, L=L)
    soft = O.Model(6, lik="analytic", analytic=t, lower=t["lower"], upper=upper, mu=mean, L=L, pen_w=w)
    z_in = -np.abs(np.random.default_rng(0).normal(size=(5, 6)))  # x_0 below its bound
    z_in[:, 0] = -np.abs(z_in[:, 0]) - 0.01
    a, ga = hard.logpost(z_in)
    b, gb = soft.logpost(z_in)
    assert np.array_equal(a, b) and np.array_equal(ga, gb)
    # on the two sides of the bound the values meet (continuity) and so do the gradients (C1)
    zb = np.zeros((1, 6))
    eps = 1e-9
    zl, zr = zb.copy(), zb.copy()
    zl[0, 0] -= eps / L[0, 0]
    zr[0, 0] += eps / L[0, 0]
    (vl, gl), (vr, gr) = soft.logpost(zl), soft.logpost(zr)
    assert abs(vl[0] - vr[0]) < 1e-6 and np.allclose(gl, gr, atol=1e-5)
    assert hard.logpost(zr, grad=False)[0] == -np.inf


def test_bounds_penalty_gradient_finite_differences():
    t, mean, cov = _linear_problem()
    L = np.linalg.cholesky(cov)
    upper = t["upper"].copy()
    upper[[0, 3]] = mean[[0, 3]]
    lower = t["lower"].copy()
    lower[2] = mean[2] + 0.5 * np.sqrt(cov[2, 2])  # dim 2's lower bound above the mean
    w = np.array([0.3, 1.0, 0.02, 0.5, 1.0, 1.0]) * np.sqrt(np.diag(cov))
    m = O.Model(6, lik="analytic", analytic=t, lower=lower, upper=upper, mu=mean, L=L, pen_w=w)
    rng = np.random.default_rng(3)
    for _ in range(4):
        z = rng.normal(size=6) * 1.5
        _, g = m.logpost(z)
        h = 1e-6
        fd = np.array([(m.logpost(z + h * np.eye(6)[j], grad=False)[0] -
                        m.logpost(z - h * np.eye(6)[j], grad=False)[0]) / (2 * h) for j in range(6)])
        assert np.allclose(g[0], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


@pytest.mark.parametrize("kernel,eps,steps,extra,wfac", [("mala", 0.5, 4000, {}, 1.0),
                                                        ("hmc", 0.35, 1500, {"n_leapfrog": 6}, 1.0),
                                                        ("mala", 0.3, 6000, {}, 0.2)])
def test_bounds_penalty_closed_form_marginal_mean(kernel, eps, steps, extra, wfac):
    """Linear 6-D target (exactly Gaussian posterior), upper bound of dim 0 at its posterior mean
    with penalty width w = wfac sd_0: the sampled mean of x_0 equals the closed form of
    _penalised_marginal_mean (w = sd_0: a half-normal joined to a narrower one; w = 0.2 sd_0:
    nearer the truncated half-normal mean mu - sd sqrt(2 / pi))."""
    t, mean, cov = _linear_problem()
    Lp = np.linalg.cholesky(cov)
    sd0 = np.sqrt(cov[0, 0])
    upper = t["upper"].copy()
    upper[0] = mean[0]
    w = np.full(6, 1.0)
    w[0] = wfac * sd0
    m = O.Model(6, lik="analytic", analytic=t, lower=t["lower"], upper=upper, mu=mean, L=Lp, pen_w=w)
    z0 = S.chains_init(128, 6, seed=7)
    z0[:, 0] = -np.abs(z0[:, 0])
    r = O.run(m, kernel, z0, eps=eps, n_steps=steps, seed=5, **extra)
    x0 = r["samples"][steps // 5:, :, 0]
    cm = x0.mean(axis=0)
    se = cm.std(ddof=1) / np.sqrt(len(cm))
    want = _penalised_marginal_mean(mean[0], sd0, w[0])
    assert abs(cm.mean() - want) < 5 * se, (cm.mean() - want) / se
    # and it differs from the unpenalised mean by many standard errors (the penalty acts)
    assert abs(cm.mean() - mean[0]) > 10 * se
