"""Pins of the oracle's convergence metrics (paper Sec. 4.1: multivariate R - 1, quantiles and the
credible metric, the 1-D Wasserstein-1 distance and the sliced Wasserstein distance) and of the
initial walker positions (Sec. 3.1)."""
import numpy as np
import pytest

import oracle as O


def test_one_dimension_worked_example():
    # chains (0, 2) and (4, 6): chain means 1 and 5, B = 8 (chains - 1 denominator); chain
    # variances 2 and 2, W = 2; R - 1 = B / W = 4
    x = np.array([[[0.0], [4.0]], [[2.0], [6.0]]])  # [draws][chains][d]
    assert O.r_minus_1(x) == pytest.approx(4.0, rel=1e-14)


def test_two_dimension_worked_example():
    # chain a: (0,0) (2,0) (0,2) (2,2); chain b: (4,1) (6,1) (4,3) (6,3)
    # means (1,1) and (5,2): B = [[8, 2], [2, 0.5]] (rank one, eigenvalues 8.5 and 0)
    # each chain: variances 4/3, no cross term: W = 4/3 I; R - 1 = 8.5 * 3/4 = 6.375
    a = np.array([[0, 0], [2, 0], [0, 2], [2, 2]], float)
    b = np.array([[4, 1], [6, 1], [4, 3], [6, 3]], float)
    x = np.stack([a, b], axis=1)
    assert O.r_minus_1(x) == pytest.approx(6.375, rel=1e-13)


def test_equal_chain_means_give_zero_and_constant_dimension_gives_nan():
    rng = np.random.default_rng(0)
    base = rng.normal(size=(50, 1, 3))
    x = np.concatenate([base, base[::-1]], axis=1)  # two chains, same draws reversed: same means
    with np.errstate(invalid="ignore", divide="ignore"):
        assert np.isnan(O.r_minus_1(x))  # B = 0: D is singular
    y = rng.normal(size=(40, 6, 3))
    y[:, :, 2] = 1.5  # a dimension with no spread at all
    with np.errstate(invalid="ignore", divide="ignore"):
        assert np.isnan(O.r_minus_1(y))


def test_affine_invariance_and_chain_order():
    # x -> A x + c maps W -> A W A^T and B -> A B A^T, so W^-1 B and the statistic are unchanged;
    # the order of the chains does not enter
    rng = np.random.default_rng(3)
    n, M, d = 60, 9, 4
    x = rng.normal(size=(n, M, d)) + rng.normal(size=(1, M, d)) * 0.3
    A = rng.normal(size=(d, d)) + 2 * np.eye(d)
    c = rng.normal(size=d)
    r0 = O.r_minus_1(x)
    assert r0 > 0
    assert O.r_minus_1(x @ A.T + c) == pytest.approx(r0, rel=1e-9)
    assert O.r_minus_1(x[:, rng.permutation(M), :]) == pytest.approx(r0, rel=1e-12)


def test_well_mixed_chains_tend_to_zero():
    # i.i.d. draws: B ~ W / n, so R - 1 shrinks like 1 / n
    rng = np.random.default_rng(5)
    r_short = O.r_minus_1(rng.normal(size=(100, 20, 3)))
    r_long = O.r_minus_1(rng.normal(size=(10000, 20, 3)))
    assert r_long < r_short and r_long < 0.01


def test_quantiles_of_an_arithmetic_sequence():
    # the 101 draws 0, 1, ..., 100: the q-quantile is 100 q exactly (rank (N - 1) q); a second
    # dimension holding 2 x + 1 has quantiles 200 q + 1
    v = np.arange(101.0)
    x = np.stack([v, 2 * v + 1], axis=-1).reshape(101, 1, 2)
    q = [0.025, 0.16, 0.5, 0.84, 0.975]
    out = O.quantiles(x, q)
    assert np.allclose(out[0], 100 * np.array(q), rtol=0, atol=1e-12)
    assert np.allclose(out[1], 200 * np.array(q) + 1, rtol=0, atol=1e-12)


def test_credible_metric_worked_example():
    # draws 0..100: the 68 % limits are 16 and 84; against true limits 20 and 80 the metric is
    # (|84 - 80| + |16 - 20|) / (80 - 20) = 8 / 60
    x = np.arange(101.0).reshape(101, 1, 1)
    cm = O.credible_metric(x, 0.68, [20.0], [80.0])
    assert cm[0] == pytest.approx(8.0 / 60.0, rel=1e-12)
    # exact limits give zero; scaling draws and limits together leaves the metric unchanged
    assert O.credible_metric(x, 0.68, [16.0], [84.0])[0] == pytest.approx(0.0, abs=1e-12)
    assert O.credible_metric(3 * x, 0.68, [60.0], [240.0])[0] == pytest.approx(8.0 / 60.0, rel=1e-12)


def test_initial_positions_of_each_strategy():
    """Sec. 3.1 initialisation strategies: repeated = the centre exactly; uniform draws inside
    the box with the uniform law's mean and variance; Gaussian draws with covariance Lc Lc^T."""
    n, d = 20000, 3
    c = np.array([0.5, -1.0, 2.0])
    rep = O.draw_positions(O.INIT_REPEATED, 7, 5, d, center=c)
    assert np.array_equal(rep, np.tile(c, (5, 1)))
    lo, hi = np.array([-3.0, 0.0, 1.0]), np.array([3.0, 1.0, 5.0])
    u = O.draw_positions(O.INIT_UNIFORM, 7, n, d, lower=lo, upper=hi)
    assert np.all(u > lo) and np.all(u < hi)
    se = (hi - lo) / np.sqrt(12 * n)
    assert np.all(np.abs(u.mean(axis=0) - (lo + hi) / 2) < 5 * se)
    assert np.allclose(u.var(axis=0), (hi - lo) ** 2 / 12, rtol=0.05)
    Lc = np.array([[1.0, 0, 0], [0.5, 2.0, 0], [-0.3, 0.2, 0.5]])
    g = O.draw_positions(O.INIT_GAUSSIAN, 7, n, d, center=c, Lc=Lc)
    assert np.allclose(g.mean(axis=0), c, atol=5 * np.sqrt(np.diag(Lc @ Lc.T) / n))
    assert np.allclose(np.cov(g, rowvar=False), Lc @ Lc.T, atol=0.08)
    # a chain's draw depends on the seed and on its index only
    assert np.array_equal(O.draw_positions(O.INIT_UNIFORM, 7, 3, d, lower=lo, upper=hi), u[:3])


def test_w1_worked_examples():
    # equal sizes: mean |sorted difference|
    assert O.w1_1d([0.0, 3.0], [1.0, 1.0]) == pytest.approx((1.0 + 2.0) / 2, rel=1e-15)
    # {0, 1} against {0, 0.5, 1}: the quantile functions differ by 1/2 on (1/3, 2/3): 1/6
    assert O.w1_1d([0.0, 1.0], [0.0, 0.5, 1.0]) == pytest.approx(1.0 / 6.0, rel=1e-14)
    # a shift by c moves every quantile by c
    x = np.random.default_rng(1).normal(size=37)
    assert O.w1_1d(x, x + 0.75) == pytest.approx(0.75, rel=1e-12)
    # symmetric, zero on identical samples
    y = np.random.default_rng(2).normal(size=53)
    assert O.w1_1d(x, y) == pytest.approx(O.w1_1d(y, x), rel=1e-12)
    assert O.w1_1d(y, y[::-1]) == 0.0


def test_sliced_wasserstein_of_a_shift_and_of_identical_sets():
    rng = np.random.default_rng(3)
    P = rng.normal(size=(400, 4))
    c = np.array([0.5, -1.0, 0.0, 2.0])
    U = O.swd_directions(9, 64, 4)
    assert np.allclose(np.linalg.norm(U, axis=1), 1.0)
    # a shift by c: every projected quantile moves by c.u, so the distance is mean |c.u|
    assert O.sliced_wasserstein(P, P + c, n_proj=64, seed=9) == pytest.approx(np.mean(np.abs(U @ c)), rel=1e-10)
    assert O.sliced_wasserstein(P, P[::-1], n_proj=64, seed=9) == pytest.approx(0.0, abs=1e-15)
    # directions uniform on the sphere S^3: E|u_i| = Gamma(2) / (sqrt(pi) Gamma(5/2)) = 4 / (3 pi)
    big = O.swd_directions(9, 4000, 4)
    assert np.abs(big).mean(axis=0) == pytest.approx(np.full(4, 4.0 / (3.0 * np.pi)), rel=0.04)


def test_w1_against_scipy_for_unequal_sizes():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(4)
    for na, nb in [(1, 1), (5, 3), (64, 100), (257, 31)]:
        a, b = rng.normal(size=na), rng.gamma(2.0, size=nb)
        assert O.w1_1d(a, b) == pytest.approx(scipy_stats.wasserstein_distance(a, b), rel=1e-12)


def test_w1_equal_sizes_is_mean_sorted_difference_and_matches_transport_lp():
    """Equal sizes: the mean absolute difference of the sorted samples (Sec. 4.1).  Unequal tiny
    sizes: the optimal-transport linear program solved by brute force (scipy's LP solver)."""
    rng = np.random.default_rng(5)
    a, b = rng.normal(size=64), rng.exponential(size=64)
    assert O.w1_1d(a, b) == pytest.approx(np.mean(np.abs(np.sort(a) - np.sort(b))), rel=1e-13)
    optimize = pytest.importorskip("scipy.optimize")
    a, b = rng.normal(size=4), rng.normal(size=6) + 0.4
    na, nb = len(a), len(b)
    cost = np.abs(a[:, None] - b[None, :]).ravel()
    A_eq = np.zeros((na + nb, na * nb))
    for i in range(na):
        A_eq[i, i * nb:(i + 1) * nb] = 1.0
    for j in range(nb):
        A_eq[na + j, j::nb] = 1.0
    b_eq = np.concatenate([np.full(na, 1.0 / na), np.full(nb, 1.0 / nb)])
    lp = optimize.linprog(cost, A_eq=A_eq, b_eq=b_eq, bounds=(0, None), method="highs")
    assert lp.success
    assert O.w1_1d(a, b) == pytest.approx(lp.fun, rel=1e-9)
