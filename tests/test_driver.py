"""The burn-in driver's host logic with a stand-in sampler (no GPU): dual averaging finds the
step size of the target acceptance on a known acceptance curve, and the burn-in runs the
adaptation protocol in order."""
import numpy as np
import pytest

from paper_2606_04895_gb300 import driver


class FakeSampler:
    """acceptance statistic exp(-eps / 0.5): 0.65 at eps = -0.5 log 0.65"""

    def __init__(self):
        self.calls = []

    def step(self, kernel, n_steps, *, eps, stats=True, **kw):
        self.calls.append(("step", n_steps, eps))
        return {"accept_stat": float(np.exp(-eps / 0.5))} if stats else None

    def welford_reset(self):
        self.calls.append(("welford_reset",))

    def adapt_cov(self, jitter0=1e-10):
        self.calls.append(("adapt_cov", jitter0))
        return np.zeros(2), np.eye(2), jitter0


def test_dual_averaging_reaches_the_target_acceptance():
    s = FakeSampler()
    eps = driver.dual_average_eps(s, "mala", 1.0, n_iter=200, chunk=10, target=0.65)
    assert eps == pytest.approx(-0.5 * np.log(0.65), rel=0.05)
    assert len(s.calls) == 200 and all(c[1] == 10 for c in s.calls)


def test_burn_in_runs_the_protocol_in_order():
    s = FakeSampler()
    eps, hist = driver.burn_in(s, "mala", eps0=0.3, n_iter=3, adapt_steps=400, chunk=40, cov_steps=500)
    kinds = [c[0] for c in s.calls]
    # per iteration: 10 adaptation chunks, reset, the accumulation steps, adaptation; then 10 chunks
    one = ["step"] * 10 + ["welford_reset", "step", "adapt_cov"]
    assert kinds == one * 3 + ["step"] * 10
    assert [c[1] for c in s.calls if c[0] == "step" and c[1] == 500] == [500, 500, 500]
    assert len(hist) == 3 and all(h["jitter"] == 1e-10 for h in hist)
    assert 0.1 < eps < 0.4


def test_burn_in_with_pooled_callbacks():
    s = FakeSampler()
    seen = []
    eps, hist = driver.burn_in(s, "mala", n_iter=1, adapt_steps=80, chunk=40, cov_steps=10,
                               adapt_cov=lambda smp: seen.append("pooled"),
                               mean_accept=lambda st, chunk: 0.65)
    assert seen == ["pooled"] and hist[0]["jitter"] is None
    assert not any(c[0] == "adapt_cov" for c in s.calls)


def test_initial_whitening_is_the_box_centre_and_scaled_widths():
    mu, L = driver.initial_whitening([-1.0, 0.0, 10.0], [3.0, 0.5, 30.0], frac=0.25)
    assert np.array_equal(mu, [1.0, 0.25, 20.0])
    assert np.array_equal(L, np.diag([1.0, 0.125, 5.0]))
    with pytest.raises(ValueError):
        driver.initial_whitening([0.0, 1.0], [1.0, 1.0])
    with pytest.raises(ValueError):
        driver.initial_whitening([0.0], [1.0], frac=0.0)


def test_aies_burn_in_is_one_long_run_in_bounded_launches():
    s = FakeSampler()
    s.step = lambda kernel, n, stats=True, **kw: s.calls.append((kernel, n, stats))
    assert driver.aies_burn_in(s, 20000, chunk=6000) == 20000
    assert s.calls == [("aies", 6000, False)] * 3 + [("aies", 2000, False)]
    assert driver.aies_burn_in(s, 0) == 0
    with pytest.raises(ValueError):
        driver.burn_in(FakeSampler(), "aies")
