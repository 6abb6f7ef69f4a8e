"""Pins for the oracle's Philox4x32-10 draws and bfloat16 rounding.

The generator is pinned by the published known-answer vectors of Salmon et al.
(tests/golden/philox4x32_10_kat.txt), by agreement with an independent
implementation (triton.language's philox, run by the Triton interpreter on the
CPU) on random counters and keys, by distributional tests and by the
counter/key structure the draws must have."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(v, 16) for v in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    rows = kat_vectors()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert [int(v) for v in O.philox4x32_10(ctr, key)] == want, (ctr, key)


_TRITON_PHILOX = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def kern(c_ptr, k_ptr, o_ptr, n, BLOCK: tl.constexpr):
    i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    m = i < n
    c = [tl.load(c_ptr + 4 * i + j, mask=m).to(tl.uint32) for j in range(4)]
    k0 = tl.load(k_ptr + 2 * i, mask=m).to(tl.uint32)
    k1 = tl.load(k_ptr + 2 * i + 1, mask=m).to(tl.uint32)
    r = tl.philox_impl(c[0], c[1], c[2], c[3], k0, k1, 10)
    for j in range(4):
        tl.store(o_ptr + 4 * i + j, r[j].to(tl.int64) & 0xffffffff, mask=m)

c, k = json.loads(sys.stdin.read())
c = torch.tensor(c, dtype=torch.int64)
k = torch.tensor(k, dtype=torch.int64)
o = torch.zeros_like(c)
kern[(triton.cdiv(len(c), 64),)](c, k, o, len(c), BLOCK=64)
print(json.dumps(o.tolist()))
"""


def test_philox_matches_an_independent_implementation():
    """Random counters and keys: the oracle's words equal triton.language's philox (a
    separate implementation of the same published generator) on every word."""
    pytest.importorskip("triton")
    import json
    rng = np.random.default_rng(17)
    ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64)
    key = rng.integers(0, 2**32, size=(256, 2), dtype=np.uint64)
    ctr[:8, 1:] = 0  # small counters as the samplers use them
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps([ctr.tolist(), key.tolist()]),
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr.strip().splitlines()[-1] if r.stderr else "")
    ref = np.array(json.loads(r.stdout), dtype=np.uint64)
    ours = np.array([[int(v) for v in O.philox4x32_10(c, k)] for c, k in zip(ctr.tolist(), key.tolist())],
                    dtype=np.uint64)
    assert np.array_equal(ours, ref)


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


@pytest.mark.parametrize("v", [0.0, 1.0, -1.0, 1.0 + 2.0**-11, 1.0 + 3 * 2.0**-11, 65504.0, 65519.9, 65520.0,
                               -70000.0, 2.0**-14, 2.0**-14 * 0.75, 2.0**-24, 2.0**-25, 3 * 2.0**-26, 1e-9,
                               0.1, -0.3, 1234.5678])
def test_fp16_round_matches_numpy(v):
    """binary16 rounding (ties to even, subnormals, overflow to inf) against numpy's conversion."""
    ref = float(np.float64(v).astype(np.float16))
    got = O.fp16_round(v)
    assert got == ref or (np.isinf(got) and np.isinf(ref) and np.sign(got) == np.sign(ref)), (v, got, ref)


def test_fp16_round_random_against_numpy_and_torch():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(6000) * np.exp(rng.uniform(-20, 12, 6000))
    ref = x.astype(np.float16).astype(np.float64)
    got = np.array([O.fp16_round(float(v)) for v in x])
    assert np.array_equal(got, ref)
    f32 = x.astype(np.float32)
    t = torch.from_numpy(f32).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(np.array([O.fp16_round(float(v)) for v in f32]), t)
