"""Pins for covariance adaptation (paper Sec. 3.2), emulator training and the
multi-chain ESS: numpy.cov / numpy.linalg.cholesky (library routines), the
Chan-merge identity, finite differences of the training loss, Adam's first
step in closed form, and the ESS of i.i.d. and AR(1) chains."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def test_pooled_cov_matches_numpy():
    x = np.random.default_rng(0).normal(size=(500, 7)) @ np.random.default_rng(1).normal(size=(7, 7))
    mean, cov = O.pooled_cov(x)
    assert np.allclose(mean, x.mean(axis=0), rtol=1e-13)
    assert np.allclose(cov, np.cov(x.T), rtol=1e-12)


def test_chan_merge_equals_single_pass():
    x = np.random.default_rng(2).normal(size=(300, 5)) + 10.0
    a, b = x[:110], x[110:]
    ma, ca = O.pooled_cov(a)
    mb, cb = O.pooled_cov(b)
    n, m, M2 = O.chan_merge(len(a), ma, ca * (len(a) - 1), len(b), mb, cb * (len(b) - 1))
    mm, cc = O.pooled_cov(x)
    assert n == len(x)
    assert np.allclose(m, mm, rtol=1e-13)
    assert np.allclose(M2 / (n - 1), cc, rtol=1e-12)


def test_cholesky_matches_numpy_and_jitter():
    A = np.random.default_rng(3).normal(size=(27, 27))
    Sg = A @ A.T + 1e-3 * np.eye(27)
    rc, L, used = O.cholesky_jitter(Sg)
    assert rc == 0 and used == 0.0
    assert np.allclose(L, np.linalg.cholesky(Sg), rtol=1e-10, atol=1e-12)
    # rank-deficient covariance (fewer samples than dims) needs the diagonal loading
    x = np.random.default_rng(4).normal(size=(5, 8))
    _, Sd = O.pooled_cov(x)
    rc, L, used = O.cholesky_jitter(Sd, 1e-10)
    assert rc == 0 and used > 0
    assert np.allclose(L @ L.T, Sd + used * np.trace(Sd) / 8 * np.eye(8), rtol=1e-9, atol=1e-12)
    # indefinite matrix: no jitter up to 1e-2 rescues it
    Bad = np.diag([1.0, 1.0, -5.0])
    rc, _, _ = O.cholesky_jitter(Bad, 1e-10)
    assert rc == -1


def test_remap_keeps_x():
    rng = np.random.default_rng(5)
    d = 6
    L0 = np.tril(rng.normal(size=(d, d))) + 3 * np.eye(d)
    L1 = np.tril(rng.normal(size=(d, d))) + 2 * np.eye(d)
    mu0, mu1 = rng.normal(size=d), rng.normal(size=d)
    z = rng.normal(size=(20, d))
    z1 = O.remap_z(mu0, L0, mu1, L1, z)
    assert np.allclose(mu0 + z @ L0.T, mu1 + z1 @ L1.T, rtol=1e-12, atol=1e-12)


def test_training_gradient_finite_differences():
    d, D, w = 4, 3, 16
    e = S.emulator(d, width=w, depth=D, seed=1)
    P = e["params"]
    X = np.random.default_rng(0).uniform(-3, 3, (9, d))
    y = np.random.default_rng(1).normal(size=9) * 5 + 20
    args = (d, D, w)
    loss, g = O.train_loss_grad(*args, P, e["in_m"], e["in_s"], 18.0, 4.0, X, y)
    rng = np.random.default_rng(2)
    idx = rng.choice(P.size, 40, replace=False)
    for i in idx:
        h = 1e-6
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        lp, _ = O.train_loss_grad(*args, Pp, e["in_m"], e["in_s"], 18.0, 4.0, X, y)
        lm, _ = O.train_loss_grad(*args, Pm, e["in_m"], e["in_s"], 18.0, 4.0, X, y)
        assert g[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_training_loss_is_mse_on_standardised_chi2():
    """All weights zero except b_o: out = b_o, so loss = mean((b_o - y_std)^2)."""
    d, D, w = 3, 2, 8
    e = S.emulator(d, width=w, depth=D, seed=1)
    P = np.zeros_like(e["params"]); P[-1] = 0.4
    X = np.random.default_rng(0).normal(size=(6, d))
    y = np.arange(6.0)
    loss, g = O.train_loss_grad(d, D, w, P, e["in_m"], e["in_s"], 1.0, 2.0, X, y)
    ys = (y - 1.0) / 2.0
    assert loss == pytest.approx(np.mean((0.4 - ys) ** 2), rel=1e-14)
    assert g[-1] == pytest.approx(2 * np.mean(0.4 - ys), rel=1e-14)


def test_training_loss_log_output():
    """Log output: the regression target is (log(chi2 - floor) - out_m) / out_s; with every weight
    zero but b_o the loss is the mean squared difference to it, and the gradient of b_o is twice
    the mean residual.  Labels below the floor are clamped to 1e-30 above it."""
    d, D, w = 3, 2, 8
    e = S.emulator(d, width=w, depth=D, seed=1)
    P = np.zeros_like(e["params"]); P[-1] = 0.4
    X = np.random.default_rng(0).normal(size=(6, d))
    y = np.array([5.0, 7.0, 12.0, 100.0, 4.5, 3.0])
    loss, g = O.train_loss_grad(d, D, w, P, e["in_m"], e["in_s"], 1.0, 2.0, X, y, out_log=1, out_floor=4.0)
    ys = (np.log(np.maximum(y - 4.0, 1e-30)) - 1.0) / 2.0
    assert loss == pytest.approx(np.mean((0.4 - ys) ** 2), rel=1e-14)
    assert g[-1] == pytest.approx(2 * np.mean(0.4 - ys), rel=1e-14)


def test_training_gradient_finite_differences_log_output():
    d, D, w = 4, 3, 16
    e = S.emulator(d, width=w, depth=D, seed=1)
    P = e["params"]
    X = np.random.default_rng(0).uniform(-3, 3, (9, d))
    y = np.random.default_rng(1).normal(size=9) * 5 + 30
    kw = dict(out_log=1, out_floor=12.0)
    loss, g = O.train_loss_grad(d, D, w, P, e["in_m"], e["in_s"], 2.5, 0.5, X, y, **kw)
    idx = np.random.default_rng(2).choice(P.size, 30, replace=False)
    for i in idx:
        h = 1e-6
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        lp, _ = O.train_loss_grad(d, D, w, Pp, e["in_m"], e["in_s"], 2.5, 0.5, X, y, **kw)
        lm, _ = O.train_loss_grad(d, D, w, Pm, e["in_m"], e["in_s"], 2.5, 0.5, X, y, **kw)
        assert g[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_training_bf16_mode_is_a_bf16_sized_perturbation():
    """The BF16 mixed-precision training mode rounds only the operands of the hidden-layer
    products: its loss equals the exact loss to BF16 accuracy and its gradient differs from the
    exact gradient by a BF16-sized amount (neither zero nor of the gradient's own size); a
    one-hidden-layer network (depth 1) has no hidden-layer product, so there it is exact."""
    d, D, w = 4, 3, 32
    e = S.emulator(d, width=w, depth=D, seed=2)
    X = np.random.default_rng(0).uniform(-3, 3, (17, d))
    y = np.random.default_rng(1).normal(size=17) * 5 + 20
    l0, g0 = O.train_loss_grad(d, D, w, e["params"], e["in_m"], e["in_s"], 18.0, 4.0, X, y)
    l1, g1 = O.train_loss_grad(d, D, w, e["params"], e["in_m"], e["in_s"], 18.0, 4.0, X, y, bf16=True)
    assert abs(l1 - l0) < 1e-2 * abs(l0)
    rel = np.max(np.abs(g1 - g0)) / np.max(np.abs(g0))
    assert 1e-5 < rel < 3e-2, rel
    e1 = S.emulator(d, width=w, depth=1, seed=2)
    a0, h0 = O.train_loss_grad(d, 1, w, e1["params"], e1["in_m"], e1["in_s"], 18.0, 4.0, X, y)
    a1, h1 = O.train_loss_grad(d, 1, w, e1["params"], e1["in_m"], e1["in_s"], 18.0, 4.0, X, y, bf16=True)
    assert a0 == a1 and np.array_equal(h0, h1)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m1, m2 = O.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-2, eps=1e-8)
    # bias-corrected first step: m_hat = g, v_hat = g^2  ->  p - lr g / (|g| + eps)
    assert np.allclose(p1, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-13)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_adam_training_reduces_loss():
    d, D, w = 3, 2, 16
    e = S.emulator(d, width=w, depth=D, seed=3)
    X = np.random.default_rng(0).uniform(-3, 3, (64, d))
    y = (X ** 2).sum(axis=1)
    P = e["params"].copy()
    m1 = np.zeros_like(P); m2 = np.zeros_like(P)
    l0 = None
    for t in range(1, 201):
        loss, g = O.train_loss_grad(d, D, w, P, e["in_m"], e["in_s"], 9.0, 5.0, X, y)
        l0 = loss if l0 is None else l0
        P, m1, m2 = O.adam(P, g, m1, m2, t, lr=1e-2)
    assert loss < 0.2 * l0


def test_ess_iid_and_ar1():
    rng = np.random.default_rng(0)
    n, M = 2000, 16
    iid = rng.normal(size=(n, M, 2))
    ess = O.ess(iid)
    assert np.all(np.abs(ess / (n * M) - 1) < 0.15)
    phi = 0.8
    x = np.zeros((n, M, 1))
    x[0] = rng.normal(size=(M, 1)) / np.sqrt(1 - phi ** 2)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + rng.normal(size=(M, 1))
    ess = O.ess(x)[0]
    assert abs(ess / (n * M) / ((1 - phi) / (1 + phi)) - 1) < 0.2
