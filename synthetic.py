"""Seeded synthetic inputs shared by the tests, the benchmark and the CUDA path.

This module only draws and assembles inputs; it evaluates no likelihood,
gradient or sampler step of the method.  It stands in for the paper's data
(Planck 2018 + BAO likelihoods behind the CLiENT emulators, Sec. 4), which are
not available: every target is a seeded random "theory map"

    f(theta) = A tanh(B theta_c + c) + N theta_n,   data = f(theta*) + sigma xi,

with A, B, c, N drawn i.i.d. N(0, 1/fan_in), and every emulator is a seeded
tanh MLP.  The three shapes are

  * 6-D  (LCDM-shaped):  B 32x6,  A 256x32, sigma 0.1, box [-3, 3]^6;
  * 8-D  (sterile-shaped): B 32x8 whose last two columns are scaled by 0.1, so
    those two directions are weakly constrained and plateau-like;
  * 27-D (nuisance-extended): 6 tanh dims + 21 linear nuisance dims with N(0,1)
    priors, A 2048x32, N 2048x21.

The data vector and the Laplace covariance used to place the truth and to draw
training inputs are part of the input recipe: they decide WHICH target is
sampled, and no test checks them.
"""
from __future__ import annotations

import numpy as np

BOX = 3.0


def _normal(rng, shape, fan_in):
    return rng.standard_normal(shape) / np.sqrt(fan_in)


def theory_map(d, *, d_c=None, n_hidden=32, n_data=256, sterile_scale=None, seed=0):
    """A, B, c (and N for d > d_c) drawn i.i.d. N(0, 1/fan_in) from ``seed``."""
    d_c = d if d_c is None else d_c
    rng = np.random.default_rng(seed)
    B = _normal(rng, (n_hidden, d_c), d_c)
    c = _normal(rng, (n_hidden,), d_c)
    A = _normal(rng, (n_data, n_hidden), n_hidden)
    N = _normal(rng, (n_data, d - d_c), d - d_c) if d > d_c else None
    if sterile_scale is not None:
        B[:, -2:] *= sterile_scale
    return {"A": A, "B": B, "c": c, "N": N, "d_c": d_c}


def _jacobian(tm, theta, linear):
    """Jacobian of the theory map at theta (input recipe only)."""
    d_c = tm["d_c"]
    a = tm["B"] @ theta[:d_c] + tm["c"]
    dt = np.ones_like(a) if linear else 1.0 - np.tanh(a) ** 2
    J = tm["A"] @ (dt[:, None] * tm["B"])
    if tm["N"] is not None:
        J = np.concatenate([J, tm["N"]], axis=1)
    return J


def _theory(tm, theta, linear):
    d_c = tm["d_c"]
    a = tm["B"] @ theta[:d_c] + tm["c"]
    f = tm["A"] @ (a if linear else np.tanh(a))
    if tm["N"] is not None:
        f = f + tm["N"] @ theta[d_c:]
    return f


def laplace_cov(tm, theta, sigma, linear=False, gauss=None):
    """sigma^2 (J^T J + prior precision)^-1 at theta (input recipe only)."""
    J = _jacobian(tm, theta, linear)
    P = J.T @ J / sigma**2
    if gauss is not None:
        P = P + np.diag(np.asarray(gauss, dtype=float))
    return np.linalg.inv(P)


def target(d=6, *, linear=False, seed=0, sigma=0.1, n_data=None, sterile=None, nuisance=False):
    """Full analytic target: theory map, truth theta*, data vector and prior.

    d=6 and d=8 use the 6-D / 8-D recipes; ``nuisance=True`` gives the 27-D one.
    The truth is redrawn until every |theta*_i| <= 3 - 6 sigma_post,i so the
    box truncates a negligible part of the posterior."""
    if nuisance:
        d_c, n_data = 6, (2048 if n_data is None else n_data)
    else:
        d_c, n_data = d, (256 if n_data is None else n_data)
    if sterile is None:
        sterile = (d == 8 and not nuisance)
    tm = theory_map(d, d_c=d_c, n_data=n_data, sterile_scale=0.1 if sterile else None, seed=seed)
    gauss = np.array([0] * d_c + [1] * (d - d_c), dtype=np.int32)
    rng = np.random.default_rng(seed + 1)
    theta = None
    for _ in range(1000):
        cand = rng.standard_normal(d)
        cand[d_c:] = np.clip(cand[d_c:], -2.0, 2.0)
        sd = np.sqrt(np.diag(laplace_cov(tm, cand, sigma, linear, gauss)))
        if np.all(np.abs(cand) <= BOX - 6.0 * sd):
            theta = cand
            break
    if theta is None:
        theta = np.zeros(d)
    noise = np.random.default_rng(seed + 2).standard_normal(n_data)
    data = _theory(tm, theta, linear) + sigma * noise
    lower = np.full(d, -BOX)
    upper = np.full(d, BOX)
    if nuisance:
        lower[d_c:] = -1e30
        upper[d_c:] = 1e30
    cov = laplace_cov(tm, theta, sigma, linear, gauss)
    return {
        "d": d, "d_c": d_c, "A": tm["A"], "B": tm["B"], "c": tm["c"], "N": tm["N"],
        "data": data, "sigma": sigma, "linear": bool(linear), "theta_star": theta,
        "lower": lower, "upper": upper, "gauss": gauss, "laplace_cov": cov,
    }


def emulator(d, *, width=512, depth=4, seed=5, in_m=None, in_s=None, out_m=0.0, out_s=1.0,
             bias_scale=0.1, out_log=0, out_floor=0.0):
    """Seeded tanh-MLP weights: W_l ~ N(0, 1/fan_in), small random biases.

    Flat layout: W1[w][d] b1[w] (W_l[w][w] b_l[w])_{l=2..D} wo[w] bo."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(1, depth + 1):
        fan_in = d if l == 1 else width
        parts.append(_normal(rng, (width, fan_in), fan_in).ravel())
        parts.append(bias_scale * rng.standard_normal(width))
    parts.append(_normal(rng, (width,), width))
    parts.append(np.array([0.0]))
    params = np.concatenate(parts)
    return {
        "d": d, "depth": depth, "width": width, "params": params,
        "in_m": np.zeros(d) if in_m is None else np.asarray(in_m, float),
        "in_s": np.full(d, np.sqrt(3.0)) if in_s is None else np.asarray(in_s, float),
        "out_m": float(out_m), "out_s": float(out_s),
        "out_log": int(out_log), "out_floor": float(out_floor),
    }


def unpack_emulator(e):
    """Split the flat parameter vector into per-layer arrays (no arithmetic)."""
    d, D, w, P = e["d"], e["depth"], e["width"], e["params"]
    W, b, o = [], [], 0
    for l in range(1, D + 1):
        fan_in = d if l == 1 else w
        W.append(P[o:o + w * fan_in].reshape(w, fan_in)); o += w * fan_in
        b.append(P[o:o + w]); o += w
    wo = P[o:o + w]; o += w
    bo = float(P[o])
    return W, b, wo, bo


def pack_emulator(W, b, wo, bo):
    parts = []
    for Wl, bl in zip(W, b):
        parts += [np.asarray(Wl, float).ravel(), np.asarray(bl, float).ravel()]
    parts += [np.asarray(wo, float).ravel(), np.array([float(bo)])]
    return np.concatenate(parts)


def chains_init(n, d, *, seed=3, scale=1.0):
    """Initial whitened positions z0 ~ N(0, scale^2 I)."""
    return scale * np.random.default_rng(seed).standard_normal((n, d))


def training_inputs(tgt, n, *, seed=4, gauss_frac=0.5, gauss_scale=3.0):
    """theta for emulator training: a fraction 1 - gauss_frac U(box), gauss_frac Gaussian around
    theta* with covariance s^2 Sigma_Laplace, the Gaussian share split evenly over the widths s in
    `gauss_scale` (a number or a tuple); the config-4 recipe is half and half at 3 sigma."""
    rng = np.random.default_rng(seed)
    d = tgt["d"]
    scales = (gauss_scale,) if np.isscalar(gauss_scale) else tuple(gauss_scale)
    n_u = n - int(round(n * gauss_frac))
    lo = np.maximum(tgt["lower"], -BOX)
    hi = np.minimum(tgt["upper"], BOX)
    xu = lo + (hi - lo) * rng.random((n_u, d))
    parts = [xu]
    n_g = n - n_u
    for k, sc in enumerate(scales):
        m = n_g // len(scales) + (1 if k < n_g % len(scales) else 0)
        Lc = np.linalg.cholesky(sc ** 2 * tgt["laplace_cov"])
        parts.append(np.clip(tgt["theta_star"] + rng.standard_normal((m, d)) @ Lc.T, lo, hi))
    x = np.concatenate(parts)
    return x[rng.permutation(n)]
