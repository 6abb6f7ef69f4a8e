"""Shared set-up for the GPU parity tests: one target, its oracle model and a
library Sampler built from the same seeded inputs."""
import numpy as np
import torch

import oracle as O
import synthetic as S


def emulator_case(d=8, width=256, depth=3, seed=5, out_s=40.0, out_m=300.0):
    e = S.emulator(d, width=width, depth=depth, seed=seed, out_m=out_m, out_s=out_s)
    return e


def whitening(d, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(d, d))
    L = np.linalg.cholesky(scale ** 2 * (A @ A.T / d + 0.5 * np.eye(d)))
    mu = 0.1 * rng.normal(size=d)
    return mu, L


def make_emulator_sampler(prec, e, n, *, mu, L, lower, upper, theta0, gauss=None, seed=11, **kw):
    from paper_2606_04895_gb300 import Sampler
    d = e["d"]
    s = Sampler(d, n, precision=prec, likelihood="emulator", seed=seed, **kw)
    s.set_emulator(e["params"], e["depth"], e["width"], e["in_m"], e["in_s"], e["out_m"], e["out_s"])
    s.init_chains(theta0, lower, upper, mu=mu, L=L, gauss=gauss)
    return s


def oracle_emulator_model(e, *, mu, L, lower, upper, gauss=None, bf16=False, fp16=False):
    return O.Model(e["d"], emulator=e, lower=lower, upper=upper, gauss=gauss, mu=mu, L=L, bf16=bf16, fp16=fp16)


def rel_err(a, b, floor=1e-12):
    a = np.asarray(a, float); b = np.asarray(b, float)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor)
