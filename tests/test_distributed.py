"""Multi-process host logic of the multi-GPU path, on CPU with gloo and two ranks:
chain sharding, the rank-order Welford merge behind covariance adaptation (checked
against a single pass over all ranks' samples with numpy.cov), the pooled mean
acceptance and the gradient average.  The library's device-side merge is replaced
by the oracle's Chan merge in a stand-in sampler (test infrastructure)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_covers_every_chain_once():
    from paper_2606_04895_gb300.distributed import shard
    for n, w, m in [(4096, 1, 1), (4096, 2, 1), (4097, 3, 1), (16384, 8, 64), (256, 3, 64)]:
        spans = [shard(n, r, w, m) for r in range(w)]
        assert sum(c for _, c in spans) == n
        pos = 0
        for first, count in spans:
            assert first == pos and count % m == 0
            pos += count
        assert max(c for _, c in spans) - min(c for _, c in spans) <= m
    with pytest.raises(ValueError):
        shard(100, 0, 2, 64)


class _Stand:
    """Holds (n, mean, M2) like a handle's Welford record; merges with the oracle."""

    def __init__(self, x):
        import oracle as O
        self.O = O
        self.d = x.shape[1]
        m, c = O.pooled_cov(x)
        self.state = (float(len(x)), m, c * (len(x) - 1))
        self.merged = None

    def welford_stats(self):
        return self.state

    def welford_reset(self):
        self.merged = (0.0, np.zeros(self.d), np.zeros((self.d, self.d)))

    def welford_merge(self, n, mean, M2):
        na, ma, Ma = self.merged
        if na == 0:
            self.merged = (n, np.array(mean), np.array(M2))
        else:
            self.merged = self.O.chan_merge(na, ma, Ma, n, mean, M2)

    def adapt_cov(self, jitter0):
        n, mean, M2 = self.merged
        return mean, M2 / (n - 1), 0.0


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_04895_gb300 import distributed as D
    rng = np.random.default_rng(100 + rank)
    x = rng.normal(size=(300 + 50 * rank, 5)) @ np.diag([1, 2, 3, 4, 5]) + rank
    s = _Stand(x)
    mean, cov, _ = D.adapt_cov(s)
    acc = D.mean_accept({"accept_stat": 0.5 + 0.2 * rank}, 100 * (rank + 1), 10)
    g = torch.full((7,), float(rank + 1))
    D.average_gradients(g)
    q.put((rank, mean, cov, acc, g.numpy()))
    dist.destroy_process_group()


def test_two_rank_adaptation_and_reductions():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=120) for _ in ps], key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    xs = [np.random.default_rng(100 + r).normal(size=(300 + 50 * r, 5)) @ np.diag([1, 2, 3, 4, 5]) + r
          for r in range(2)]
    allx = np.concatenate(xs)
    for r in range(2):
        _, mean, cov, acc, g = res[r]
        assert np.allclose(mean, allx.mean(axis=0), rtol=1e-12, atol=1e-12)
        assert np.allclose(cov, np.cov(allx.T), rtol=1e-10)
        assert acc == pytest.approx((0.5 * 100 + 0.7 * 200) / 300)
        assert np.allclose(g, 1.5)
    # bit-identical on both ranks
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])


class _FakeAcceptance:
    """A stand-in sampler whose acceptance statistic falls with eps at a rank-dependent rate."""

    def __init__(self, rate, n):
        self.rate, self.n = rate, n

    def step(self, kernel, n_steps, *, eps, stats=True, **kw):
        return {"accept_stat": float(np.exp(-eps / self.rate))} if stats else None


def _driver_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_04895_gb300 import distributed as D
    from paper_2606_04895_gb300 import driver
    s = _FakeAcceptance(0.4 + 0.2 * rank, 64 * (rank + 1))
    eps = driver.dual_average_eps(s, "mala", 0.5, n_iter=150, chunk=20, target=0.65,
                                  mean_accept=lambda st, chunk: D.mean_accept(st, s.n, chunk))
    q.put((rank, eps))
    dist.destroy_process_group()


def test_two_rank_step_size_adaptation_agrees():
    """The burn-in driver's dual averaging on the acceptance statistic pooled over ranks gives
    every rank the same step size, the one of the chain-weighted mean acceptance curve."""
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_driver_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=120) for _ in ps], key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1]
    # the pooled curve (64 chains at rate 0.4, 128 at rate 0.6) crosses 0.65 at eps*
    f = lambda e: (64 * np.exp(-e / 0.4) + 128 * np.exp(-e / 0.6)) / 192 - 0.65
    lo, hi = 0.0, 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) > 0 else (lo, mid)
    assert res[0][1] == pytest.approx(lo, rel=0.06)


def _rhat_draws(rank):
    """AR(1) chains with chain offsets; rank r holds 40 + 24 r chains of 150 draws in 4-D."""
    rng = np.random.default_rng(300 + rank)
    n, M, d = 150, 40 + 24 * rank, 4
    x = np.zeros((n, M, d))
    x[0] = rng.normal(size=(M, d))
    for t in range(1, n):
        x[t] = 0.6 * x[t - 1] + rng.normal(size=(M, d))
    return x + 0.4 * rng.normal(size=(1, M, d)) + rank * 0.1


def _parts(x):
    """A handle's R - 1 part computed in numpy: chain means and within-chain cross products."""
    m = x.mean(axis=0)
    dev = x - m
    return m, np.einsum("tca,tcb->ab", dev, dev)


def _rhat_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_04895_gb300 import distributed as D
    m, S = _parts(_rhat_draws(rank))
    q.put((rank, D.pooled_r_minus_1(m, S, 150)))
    dist.destroy_process_group()


def test_two_rank_pooled_r_minus_1():
    """R - 1 over both ranks' chains (different chain counts per rank) from the gathered parts:
    the same number on both ranks, equal to the oracle's R - 1 of all draws together."""
    import oracle as O
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rhat_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=120) for _ in ps], key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1]
    allx = np.concatenate([_rhat_draws(r) for r in range(2)], axis=1)
    assert res[0][1] == pytest.approx(O.r_minus_1(allx), rel=1e-10)
