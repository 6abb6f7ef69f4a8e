"""Burn-in driver: the adaptation protocol of the paper (Sec. 3.2, and the burn-in of the
comparisons in Sec. 4) as a sequence of library calls -- step-size adaptation by dual
averaging, Welford accumulation and covariance adaptation.  Host-side sequencing only: every
step runs in the library's kernels."""
from __future__ import annotations

import numpy as np


def dual_average_eps(sampler, kernel, eps0, *, n_iter=25, chunk=40, target=0.65, mean_accept=None, **kw):
    """Step size by dual averaging on log eps (Hoffman & Gelman 2014, Sec. 3.2, with their
    gamma = 0.05, t0 = 10, kappa = 0.75, mu = log(10 eps0)): n_iter chunks of `chunk` steps, each
    driving the averaged statistic toward `target` with the mean acceptance statistic of all
    chains over the chunk (`mean_accept(stats, chunk)` replaces it, e.g. pooled over ranks).
    Returns the averaged step size."""
    mu = np.log(10.0 * eps0)
    h_bar, log_eps_bar, log_eps = 0.0, 0.0, np.log(eps0)
    gamma, t0, kappa = 0.05, 10.0, 0.75
    for m in range(1, n_iter + 1):
        st = sampler.step(kernel, chunk, eps=float(np.exp(log_eps)), **kw)
        a = st["accept_stat"] if mean_accept is None else mean_accept(st, chunk)
        h_bar = (1.0 - 1.0 / (m + t0)) * h_bar + (target - a) / (m + t0)
        log_eps = mu - np.sqrt(m) / gamma * h_bar
        eta = m ** (-kappa)
        log_eps_bar = eta * log_eps + (1.0 - eta) * log_eps_bar
    return float(np.exp(log_eps_bar))


def initial_whitening(lower, upper, frac=0.1):
    """Starting whitening of the burn-in (Sec. 4: a diagonal covariance whose scales are
    proportional to the bounding box; the factor is not given, `frac` is it): mu the box
    centre, L = diag(frac (upper - lower)).  Returns (mu, L)."""
    lo, up = np.asarray(lower, dtype=np.float64), np.asarray(upper, dtype=np.float64)
    if lo.shape != up.shape or not np.all(up > lo):
        raise ValueError("initial_whitening: need upper > lower, same shapes")
    if not frac > 0:
        raise ValueError("initial_whitening: frac must be positive")
    return 0.5 * (lo + up), np.diag(frac * (up - lo))


def aies_burn_in(sampler, n_steps=20000, *, chunk=5000, **kw):
    """AIES burn-in (Sec. 4, Sec. 4.3): no step-size or covariance adaptation, one long run
    (20,000 steps on the 27-D target) whose last walker positions start the final sampling;
    run as launches of at most `chunk` steps.  Returns the number of steps run."""
    if n_steps < 0 or chunk < 1:
        raise ValueError("aies_burn_in: need n_steps >= 0 and chunk >= 1")
    done = 0
    while done < n_steps:
        k = min(chunk, n_steps - done)
        sampler.step("aies", k, stats=False, **kw)
        done += k
    return done


def burn_in(sampler, kernel, *, eps0=0.3, n_iter=3, adapt_steps=1000, chunk=40, cov_steps=5000, target=0.65,
            jitter0=1e-10, adapt_cov=None, mean_accept=None, **kw):
    """The paper's burn-in: n_iter iterations (three; five for MALA on its sterile-neutrino
    target), each a step-size adaptation over the first `adapt_steps` steps followed by
    `cov_steps` steps whose x-space draws are accumulated (Welford) and a covariance adaptation
    (new whitening; chains keep their positions); a last step-size adaptation for the final
    sampling.  `adapt_cov(sampler)` replaces the local adaptation (e.g. pooled over ranks).
    Returns (eps, history) with one entry per iteration.  AIES has neither a step size nor a
    whitening to adapt: its burn-in is `aies_burn_in`."""
    if kernel == "aies":
        raise ValueError("burn_in: AIES adapts neither a step size nor a covariance; use aies_burn_in")
    eps, hist = float(eps0), []
    n_chunks = max(1, adapt_steps // chunk)
    for it in range(n_iter):
        eps = dual_average_eps(sampler, kernel, eps, n_iter=n_chunks, chunk=chunk, target=target,
                               mean_accept=mean_accept, **kw)
        sampler.welford_reset()
        sampler.step(kernel, cov_steps, eps=eps, stats=False, **kw)
        if adapt_cov is None:
            _, _, jitter = sampler.adapt_cov(jitter0)
        else:
            adapt_cov(sampler)
            jitter = None
        hist.append({"iteration": it, "eps": eps, "jitter": jitter})
    eps = dual_average_eps(sampler, kernel, eps, n_iter=n_chunks, chunk=chunk, target=target,
                           mean_accept=mean_accept, **kw)
    return eps, hist
