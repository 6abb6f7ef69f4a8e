"""Several GPUs, one process each: chains shard, the covariance statistics and the
step-size feedback are the exchange steps.

Chains are independent, so every rank owns a contiguous share of them and the
sampling step needs no communication (weak scaling).  Two things cross ranks:

* covariance adaptation (paper Sec. 3.2) pools the Welford statistics of every
  rank's chains: each rank reads its FP64 triple (n, mean, M2), the triples are
  all-gathered and every rank merges them in rank order with the library's
  pairwise merge, so all ranks adapt to the same whitening bit for bit;
* step-size adaptation uses the mean acceptance statistic over all chains
  (an all-reduce of two numbers);
* R - 1 over all chains (Sec. 4.1) gathers every rank's chain means and within-chain cross
  products.

Data-parallel emulator training averages the per-rank gradients
(all-reduce) before the Adam update.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard(n_total: int, rank: int, world: int, multiple: int = 1):
    """Contiguous share of n_total chains for `rank`: (first index, count).  Counts are
    multiples of `multiple` (e.g. an AIES ensemble) and differ by at most one unit."""
    units = n_total // multiple
    if units * multiple != n_total:
        raise ValueError("n_total must be a multiple of `multiple`")
    base, extra = divmod(units, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first * multiple, count * multiple


def _device_for(group):
    backend = dist.get_backend(group)
    return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")


def gather_welford(sampler, group=None):
    """All ranks' (n, mean, M2) triples, in rank order."""
    n, mean, M2 = sampler.welford_stats()
    d = len(mean)
    dev = _device_for(group)
    mine = torch.tensor(np.concatenate([[n], mean, M2.ravel()]), dtype=torch.float64, device=dev)
    world = dist.get_world_size(group)
    outs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(outs, mine, group=group)
    res = []
    for o in outs:
        v = o.cpu().numpy()
        res.append((float(v[0]), v[1:1 + d], v[1 + d:].reshape(d, d)))
    return res


def adapt_cov(sampler, jitter0=1e-10, group=None):
    """Covariance adaptation over the chains of every rank: same mu, L on all ranks."""
    triples = gather_welford(sampler, group)
    sampler.welford_reset()
    for n, mean, M2 in triples:
        sampler.welford_merge(n, mean, M2)
    return sampler.adapt_cov(jitter0)


def pooled_r_minus_1(chain_means, S, n_draws: int, group=None) -> float:
    """R - 1 (Sec. 4.1) over every rank's chains from each rank's part (its chain means and
    within-chain cross products, `Sampler.r_minus_1_parts`): the means are all-gathered in rank
    order, the cross products all-gathered and summed in rank order, so every rank computes
    the same value.  Ranks may hold different numbers of chains."""
    from . import r_minus_1_combine
    means = np.ascontiguousarray(chain_means, dtype=np.float64)
    m_local, d = means.shape
    dev = _device_for(group)
    world = dist.get_world_size(group)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([m_local], dtype=torch.int64, device=dev), group=group)
    counts = [int(c.item()) for c in counts]
    m_max = max(counts)
    mine = torch.zeros((m_max * d + d * d,), dtype=torch.float64, device=dev)
    mine[: m_local * d] = torch.as_tensor(means.ravel(), dtype=torch.float64, device=dev)
    mine[m_max * d:] = torch.as_tensor(np.asarray(S, dtype=np.float64).ravel(), dtype=torch.float64, device=dev)
    outs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(outs, mine, group=group)
    all_means, S_sum = [], np.zeros((d, d))
    for c, o in zip(counts, outs):
        v = o.cpu().numpy()
        all_means.append(v[: c * d].reshape(c, d))
        S_sum = S_sum + v[m_max * d:].reshape(d, d)
    return r_minus_1_combine(n_draws, np.concatenate(all_means), S_sum)


def mean_accept(stats: dict, n_chains_local: int, n_steps: int, group=None) -> float:
    """Mean acceptance statistic over every rank's chains for one bst_step call."""
    dev = _device_for(group)
    t = torch.tensor([stats["accept_stat"] * n_chains_local * n_steps, n_chains_local * n_steps],
                     dtype=torch.float64, device=dev)
    dist.all_reduce(t, group=group)
    return float(t[0] / t[1])


def average_gradients(grad: torch.Tensor, group=None) -> torch.Tensor:
    """In-place mean of a gradient tensor over ranks (data-parallel training)."""
    dist.all_reduce(grad, group=group)
    grad /= dist.get_world_size(group)
    return grad
