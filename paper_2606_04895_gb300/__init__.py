"""GB300 (sm_103a) batched emulator posterior sampling.

Python face of the C-ABI library ``libbst.so`` (``include/bst.h``), after
"Posterior sampling in the Age of Emulators" (arXiv 2606.04895).  The paper's
unified interface (Sec. 3.1) -- a sampler built from a log-probability and
bounds, run with a method, a number of steps and a number of chains, returning
samples, acceptance rates and evaluation counts -- is :class:`Sampler`.

Every computation runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory (tensors) and the current
CUDA stream.  There is no CPU fallback: without the built library and a CUDA
device, creating a :class:`Sampler` raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (AIES, AIES_DE, BF16, FP16, FP32, FP64, HMC, LIK_ANALYTIC, LIK_EMULATOR, MALA, MH, NUTS,
                   NUTS_MULTINOMIAL, BstError)

__all__ = ["Sampler", "Results", "BstError", "EmulatorLogL", "emulator_logl", "KERNELS", "PRECISIONS",
           "n_params", "r_minus_1_combine"]

KERNELS = {"mh": MH, "mala": MALA, "hmc": HMC, "nuts": NUTS, "aies": AIES, "aies_de": AIES_DE,
           "nuts_multinomial": NUTS_MULTINOMIAL}
PRECISIONS = {"bf16": BF16, "fp16": FP16, "fp32": FP32, "fp64": FP64}


def n_params(d, depth, width):
    return d * width + width + (depth - 1) * (width * width + width) + width + 1


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


@dataclass
class Results:
    """Return value of :meth:`Sampler.sample` (paper Sec. 3.1): samples, acceptance rate, evaluations."""
    samples: torch.Tensor
    acceptance_rate: float
    evaluations: int
    accept_stat: float
    divergences: int


class Sampler:
    """One handle of the library: n_chains chains of a d-dimensional target on one GPU."""

    def __init__(self, d, n_chains, *, precision="bf16", likelihood="emulator", seed=0, max_depth=8,
                 aies_walkers=64, aies_a=2.0, thin=1, device=0):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2606_04895_gb300 needs a CUDA device (no CPU fallback)")
        self.lib = _lib.load()
        self.d, self.n = int(d), int(n_chains)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        self.device = torch.device("cuda", device)
        cfg = _lib.Config(d=self.d, n_chains=self.n, precision=self.precision,
                          lik_kind=LIK_EMULATOR if likelihood == "emulator" else LIK_ANALYTIC,
                          seed=int(seed), max_depth=int(max_depth), aies_walkers=int(aies_walkers),
                          aies_a=float(aies_a), thin=int(thin), device=int(device))
        self.thin = int(thin)
        h = C.c_void_p()
        _lib.check(self.lib.bst_create(C.byref(h), C.byref(cfg)))
        self.h = h

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.bst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ likelihoods
    def set_emulator(self, params, depth, width, in_m, in_s, out_m=0.0, out_s=1.0, out_log=0, out_floor=0.0):
        """out_log = 1: chi2 = out_floor + exp(out_s out + out_m) (bst_set_emulator_output)."""
        P, m, s = _f64(params), _f64(in_m), _f64(in_s)
        _lib.check(self.lib.bst_set_emulator(self.h, int(depth), int(width), _p(P), _p(m), _p(s),
                                             float(out_m), float(out_s)))
        if out_log:
            _lib.check(self.lib.bst_set_emulator_output(self.h, 1, float(out_floor)))
        self.depth, self.width = int(depth), int(width)

    def get_emulator(self):
        P = np.zeros(n_params(self.d, self.depth, self.width))
        _lib.check(self.lib.bst_get_emulator(self.h, _p(P)))
        return P

    def set_analytic(self, A, B, c, data, sigma, *, d_c=None, N=None, linear=False):
        A, B, c, data = _f64(A), _f64(B), _f64(c), _f64(data)
        d_c = self.d if d_c is None else int(d_c)
        N = None if N is None else _f64(N)
        _lib.check(self.lib.bst_set_analytic(self.h, d_c, A.shape[1], A.shape[0], _p(A), _p(B), _p(c), _p(N),
                                             _p(data), float(sigma), int(bool(linear))))

    # ------------------------------------------------------------------ chains
    def init_chains(self, theta0, lower, upper, *, mu=None, L=None, gauss=None):
        th = _f64(theta0).reshape(self.n, self.d)
        lo, up = _f64(lower), _f64(upper)
        mu = _f64(np.zeros(self.d) if mu is None else mu)
        L = _f64(np.eye(self.d) if L is None else L)
        g = None if gauss is None else np.ascontiguousarray(gauss, dtype=np.int32)
        _lib.check(self.lib.bst_init_chains(self.h, _p(th), _p(lo), _p(up), _p(g), _p(mu), _p(L)))

    def step(self, kernel, n_steps, *, eps=0.1, n_leapfrog=10, samples=None, stats=True, stream=None):
        """Advance all chains n_steps iterations.  samples: optional tensor
        [n_steps // thin][n_chains][d] receiving x-space samples, on the device or in pinned
        host memory (written there by the kernel directly; read it after synchronising)."""
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        if samples is not None:
            if isinstance(samples, torch.Tensor) and not samples.is_cuda:
                if not (samples.is_pinned() and samples.dtype == self.dtype and samples.is_contiguous()):
                    raise BstError(_lib.ERR_ARG, f"expected a contiguous pinned {self.dtype} host tensor")
                if tuple(samples.shape) != (n_steps // self.thin, self.n, self.d):
                    raise BstError(_lib.ERR_ARG, f"expected shape {(n_steps // self.thin, self.n, self.d)}")
            else:
                self._check_dev(samples, (n_steps // self.thin, self.n, self.d))
        st = _lib.StepStats() if stats else None
        _lib.check(self.lib.bst_step(self.h, k, float(eps), int(n_leapfrog), int(n_steps),
                                     None if samples is None else C.c_void_p(samples.data_ptr()),
                                     _stream_ptr(stream), C.byref(st) if stats else None))
        if stats:
            return {"accepts": st.accepts, "evals": st.evals, "divergences": st.divergences,
                    "accept_stat": st.accept_stat}
        return None

    def sample(self, method, n_steps, *, eps=0.1, n_leapfrog=10):
        """Paper Sec. 3.1 call: returns samples, acceptance rate and evaluation count."""
        out = torch.empty((n_steps // self.thin, self.n, self.d), dtype=self.dtype, device=self.device)
        st = self.step(method, n_steps, eps=eps, n_leapfrog=n_leapfrog, samples=out, stats=True)
        return Results(samples=out, acceptance_rate=st["accepts"] / max(1, self.n * n_steps),
                       evaluations=st["evals"], accept_stat=st["accept_stat"], divergences=st["divergences"])

    # ------------------------------------------------------------------ likelihood calls
    def loglike(self, theta, stream=None):
        theta = self._as_dev(theta)
        m = theta.shape[0]
        out = torch.empty(m, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.bst_loglike(self.h, C.c_void_p(theta.data_ptr()), m, C.c_void_p(out.data_ptr()),
                                        _stream_ptr(stream)))
        return out

    def grad_loglike(self, theta, stream=None):
        theta = self._as_dev(theta)
        m = theta.shape[0]
        out = torch.empty(m, dtype=self.dtype, device=self.device)
        g = torch.empty((m, self.d), dtype=self.dtype, device=self.device)
        _lib.check(self.lib.bst_grad_loglike(self.h, C.c_void_p(theta.data_ptr()), m, C.c_void_p(out.data_ptr()),
                                             C.c_void_p(g.data_ptr()), _stream_ptr(stream)))
        return out, g

    # ------------------------------------------------------------------ adaptation
    def welford_reset(self):
        _lib.check(self.lib.bst_welford_reset(self.h))

    def welford_add(self, x, stream=None):
        x = self._as_dev(x)
        _lib.check(self.lib.bst_welford_add(self.h, C.c_void_p(x.data_ptr()), x.shape[0], _stream_ptr(stream)))

    def welford_stats(self):
        n = np.zeros(1); mean = np.zeros(self.d); M2 = np.zeros((self.d, self.d))
        _lib.check(self.lib.bst_welford_stats(self.h, _p(n), _p(mean), _p(M2)))
        return float(n[0]), mean, M2

    def welford_merge(self, n, mean, M2):
        mean, M2 = _f64(mean), _f64(M2)
        _lib.check(self.lib.bst_welford_merge(self.h, float(n), _p(mean), _p(M2)))

    def adapt_cov(self, jitter0=1e-10):
        mu = np.zeros(self.d)
        L = np.zeros((self.d, self.d))
        used = np.zeros(1)
        _lib.check(self.lib.bst_adapt_cov(self.h, float(jitter0), _p(mu), _p(L), _p(used)))
        return mu, L, float(used[0])

    # ------------------------------------------------------------------ state
    def get_state(self):
        z = np.zeros((self.n, self.d)); lp = np.zeros(self.n); g = np.zeros((self.n, self.d))
        it = np.zeros(self.n, dtype=np.uint32)
        _lib.check(self.lib.bst_get_state(self.h, _p(z), _p(lp), _p(g), _p(it)))
        return {"z": z, "logp": lp, "grad": g, "iter": it}

    def set_state(self, st):
        z, lp, g = _f64(st["z"]), _f64(st["logp"]), _f64(st["grad"])
        it = np.ascontiguousarray(st["iter"], dtype=np.uint32)
        _lib.check(self.lib.bst_set_state(self.h, _p(z), _p(lp), _p(g), _p(it)))

    def whitening(self):
        mu = np.zeros(self.d); L = np.zeros((self.d, self.d))
        _lib.check(self.lib.bst_get_whitening(self.h, _p(mu), _p(L)))
        return mu, L

    def counters(self):
        a = np.zeros(self.n, dtype=np.int64); e = np.zeros(self.n, dtype=np.int64)
        dv = np.zeros(self.n, dtype=np.int64); s = np.zeros(self.n)
        _lib.check(self.lib.bst_get_counters(self.h, _p(a), _p(e), _p(dv), _p(s)))
        return {"accepts": a, "evals": e, "divergences": dv, "accept_stat": s}

    # ------------------------------------------------------------------ training
    def train_step(self, X, chi2, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss_out=None, stream=None):
        X = X.contiguous().float(); y = chi2.contiguous().float()
        _lib.check(self.lib.bst_train_step(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), X.shape[0],
                                           lr, beta1, beta2, eps,
                                           None if loss_out is None else C.c_void_p(loss_out.data_ptr()),
                                           _stream_ptr(stream)))

    def train_apply(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        g = grad.contiguous().float()
        _lib.check(self.lib.bst_train_apply(self.h, C.c_void_p(g.data_ptr()), lr, beta1, beta2, eps,
                                            _stream_ptr(stream)))

    def train_grad(self, X, chi2, stream=None):
        X = X.contiguous().float(); y = chi2.contiguous().float()
        g = torch.empty(n_params(self.d, self.depth, self.width), dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _lib.check(self.lib.bst_train_grad(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), X.shape[0],
                                           C.c_void_p(g.data_ptr()), C.c_void_p(loss.data_ptr()),
                                           _stream_ptr(stream)))
        return loss, g

    # ------------------------------------------------------------------ diagnostics
    def ess(self, samples):
        self._check_dev(samples, (samples.shape[0], self.n, self.d))
        out = np.zeros(self.d)
        _lib.check(self.lib.bst_ess(self.h, C.c_void_p(samples.data_ptr()), samples.shape[0], _p(out)))
        return out

    INIT_STRATEGIES = {"repeated": 0, "uniform": 1, "gaussian": 2}

    def draw_positions(self, strategy, *, center=None, L=None, lower=None, upper=None):
        """Initial positions theta[n_chains][d] by a strategy of Sec. 3.1 ("repeated",
        "uniform" in [lower, upper], "gaussian" center + L xi), drawn on the device."""
        def arr(v, shape):
            return None if v is None else np.ascontiguousarray(v, dtype=np.float64).reshape(shape)
        c, Lc, lo, up = arr(center, self.d), arr(L, (self.d, self.d)), arr(lower, self.d), arr(upper, self.d)
        out = np.zeros((self.n, self.d))
        ptr = lambda v: None if v is None else _p(v)
        _lib.check(self.lib.bst_draw_positions(self.h, self.INIT_STRATEGIES[strategy], ptr(c), ptr(Lc), ptr(lo),
                                               ptr(up), _p(out)))
        return out

    def set_whitening(self, mu, L):
        """New whitening x = mu + L z for the chains (their x is kept; z remapped)."""
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(self.d)
        L = np.ascontiguousarray(L, dtype=np.float64).reshape(self.d, self.d)
        _lib.check(self.lib.bst_set_whitening(self.h, _p(mu), _p(L)))

    def set_bounds_penalty(self, width=None):
        """Smooth bounds (Sec. 3.1): width[d] > 0 replaces a dimension's hard box by the penalty
        factor exp(-r^2 / 2), r = distance outside the box / width; 0 keeps the hard box; None
        restores hard bounds everywhere (bst_set_bounds_penalty)."""
        w = None if width is None else _f64(np.broadcast_to(np.asarray(width, dtype=np.float64), (self.d,)))
        _lib.check(self.lib.bst_set_bounds_penalty(self.h, None if w is None else _p(w)))

    def set_step_multipliers(self, m):
        """Step sizes eps m_i along the whitened directions: the whitening L diag(m)."""
        mu, L = self.whitening()
        self.set_whitening(mu, L * np.asarray(m, dtype=np.float64)[None, :])

    def r_minus_1(self, samples):
        """Multivariate Gelman-Rubin R - 1 (Sec. 4.1) of samples[n_draws][n_chains][d] (NaN
        when undefined)."""
        self._check_dev(samples, (samples.shape[0], self.n, self.d))
        out = np.zeros(1)
        _lib.check(self.lib.bst_r_minus_1(self.h, C.c_void_p(samples.data_ptr()), samples.shape[0], _p(out)))
        return float(out[0])

    def r_minus_1_parts(self, samples):
        """This handle's share of R - 1: (chain means [n][d], pooled within-chain cross products
        S [d][d]) of samples[n_draws][n_chains][d], for `r_minus_1_combine` over several handles."""
        self._check_dev(samples, (samples.shape[0], self.n, self.d))
        means = np.zeros((self.n, self.d))
        S = np.zeros((self.d, self.d))
        _lib.check(self.lib.bst_r_minus_1_parts(self.h, C.c_void_p(samples.data_ptr()), samples.shape[0], _p(means),
                                                _p(S)))
        return means, S

    def quantiles(self, samples, q):
        """Per-dimension quantiles of the pooled draws samples[n_draws][n_chains][d]; [d][len(q)]."""
        self._check_dev(samples, (samples.shape[0], self.n, self.d))
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((self.d, q.size))
        _lib.check(self.lib.bst_quantiles(self.h, C.c_void_p(samples.data_ptr()), samples.shape[0], _p(q), q.size,
                                          _p(out)))
        return out

    def credible_metric(self, samples, alpha, true_lo, true_hi):
        """Credible metric of Sec. 4.1 per dimension against the true limits."""
        self._check_dev(samples, (samples.shape[0], self.n, self.d))
        lo = np.ascontiguousarray(true_lo, dtype=np.float64)
        hi = np.ascontiguousarray(true_hi, dtype=np.float64)
        out = np.zeros(self.d)
        _lib.check(self.lib.bst_credible_metric(self.h, C.c_void_p(samples.data_ptr()), samples.shape[0], float(alpha),
                                                _p(lo), _p(hi), _p(out)))
        return out

    def sliced_wasserstein(self, samples, reference, n_proj=500, seed=0):
        """Sliced Wasserstein distance of Sec. 4.1 between the pooled draws samples[n_draws][n][d]
        and reference[n_ref][d] (both CUDA tensors of this sampler's dtype), over n_proj
        directions fixed by `seed`."""
        self._check_dev(samples, (samples.shape[0], self.n, self.d))
        self._check_dev(reference, (reference.shape[0], self.d))
        out = C.c_double(0.0)
        _lib.check(self.lib.bst_sliced_wasserstein(self.h, C.c_void_p(samples.data_ptr()), samples.shape[0],
                                                   C.c_void_p(reference.data_ptr()), reference.shape[0], int(n_proj),
                                                   int(seed), C.byref(out)))
        return out.value

    def sync(self, stream=None):
        _lib.check(self.lib.bst_sync(self.h, _stream_ptr(stream)))

    # ------------------------------------------------------------------ helpers
    def _as_dev(self, x):
        if not isinstance(x, torch.Tensor):
            x = torch.as_tensor(np.asarray(x))
        x = x.to(device=self.device, dtype=self.dtype).contiguous()
        if x.dim() == 1:
            x = x.reshape(-1, self.d)
        return x

    def _check_dev(self, t, shape):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise BstError(_lib.ERR_ARG, f"expected a contiguous {self.dtype} CUDA tensor")
        if tuple(t.shape) != tuple(shape):
            raise BstError(_lib.ERR_ARG, f"expected shape {tuple(shape)}, got {tuple(t.shape)}")


class EmulatorLogL(torch.autograd.Function):
    """logL(theta) of a Sampler's likelihood as a differentiable torch op.

    Forward calls bst_loglike (no activations kept); backward recomputes the
    forward and runs the hand-written adjoint through bst_grad_loglike, so
    memory stays O(batch) however large the batch is."""

    @staticmethod
    def forward(ctx, theta, sampler):
        ctx.sampler = sampler
        ctx.save_for_backward(theta)
        return sampler.loglike(theta.detach())

    @staticmethod
    def backward(ctx, grad_out):
        (theta,) = ctx.saved_tensors
        _, g = ctx.sampler.grad_loglike(theta.detach())
        return grad_out.to(g.dtype)[:, None] * g, None


def r_minus_1_combine(n_draws, chain_means, S):
    """R - 1 (Sec. 4.1) from the chain means of all chains (concatenated over handles,
    [n_chains][d]) and the sum of their within-chain cross products S [d][d] (host-side
    library call; needs no device)."""
    means = np.ascontiguousarray(chain_means, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    n_chains, d = means.shape
    if S.shape != (d, d):
        raise BstError(_lib.ERR_ARG, f"S must be {d} x {d}")
    out = np.zeros(1)
    _lib.check(_lib.load().bst_r_minus_1_combine(int(n_chains), int(n_draws), int(d), _p(means), _p(S), _p(out)))
    return float(out[0])


def emulator_logl(theta, sampler):
    return EmulatorLogL.apply(theta, sampler)
