"""Pins for the oracle's Philox4x32-10 draws and bfloat16 rounding.

Philox parity with an external known-answer table is unpinned (no such table
is available); the generator is pinned by distributional tests and by the
counter/key structure the draws must have."""
import numpy as np
import pytest
import torch
from scipy import stats

import oracle as O


def test_philox_counter_and_key_sensitivity():
    base = O.philox4x32_10([0, 0, 0, 0], [0, 0])
    seen = {tuple(base)}
    for w in range(4):
        ctr = [0, 0, 0, 0]
        ctr[w] = 1
        seen.add(tuple(O.philox4x32_10(ctr, [0, 0])))
    for w in range(2):
        key = [0, 0]
        key[w] = 1
        seen.add(tuple(O.philox4x32_10([0, 0, 0, 0], key)))
    assert len(seen) == 7
    # avalanche: flipping one counter bit flips about half the 128 output bits
    flips = []
    for b in range(32):
        o = O.philox4x32_10([1 << b, 7, 9, 11], [3, 5])
        r = O.philox4x32_10([0, 7, 9, 11], [3, 5])
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(o, r)))
    assert 50 < np.mean(flips) < 78


def test_uniforms_are_uniform_on_open_interval():
    u = np.array([O.uniform(1234, c, 5, O.P_ACCEPT, k) for c in range(2000) for k in range(8)])
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    hist, _ = np.histogram(u, bins=32, range=(0, 1))
    assert stats.chisquare(hist).pvalue > 1e-4
    # lag-1 serial correlation within a block stream
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 5 / np.sqrt(u.size)


def test_uniform_grid_is_24_bit():
    u = np.array([O.uniform(7, c, 0, 1, 0) for c in range(500)])
    k = u * 2**24 - 0.5
    assert np.allclose(k, np.round(k), atol=1e-9)


def test_normals_are_standard_normal():
    x = np.concatenate([O.normals(99, c, 3, O.P_XI, 27) for c in range(1500)])
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / x.size)
    assert abs(stats.kurtosis(x)) < 5 * np.sqrt(24 / x.size)
    assert stats.kstest(x, "norm").pvalue > 1e-4


def test_normal_blocks_are_prefix_stable():
    a = O.normals(5, 17, 2, O.P_XI, 27)
    b = O.normals(5, 17, 2, O.P_XI, 8)
    assert np.array_equal(a[:8], b)


@pytest.mark.parametrize("v", [1.0, -3.0, 0.1, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5e-3, 123.456, 7e-20])
def test_bf16_round_matches_torch(v):
    f32 = float(np.float32(v))
    ref = torch.tensor(f32, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).item()
    assert O.bf16_round(f32) == ref


def test_bf16_round_random_against_torch():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(4000) * np.exp(rng.uniform(-8, 8, 4000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.bf16_round(float(v)) for v in x])
    assert np.array_equal(got, ref)
