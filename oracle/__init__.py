"""FP64 CPU oracle for batched emulator posterior sampling -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never links, loads or calls it, and it shares no code with
``paper_2606_04895_gb300/csrc``.

The C source (``oracle.c``) follows the paper ("Posterior sampling in the Age
of Emulators", arXiv 2606.04895) and the algorithms it cites; every function
there names its source.  This module compiles it with gcc and wraps it with
ctypes, converting numpy arrays to plain pointers.

Parity pins: see ``tests/test_oracle_*.py``.  The Philox generator is pinned by
the published known-answer vectors of Philox4x32-10 (``tests/golden/``) besides
its statistical and structural tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

MH, MALA, HMC, NUTS, AIES, AIES_DE, NUTS_MULTINOMIAL = 0, 1, 2, 3, 4, 5, 6
KERNELS = {"mh": MH, "mala": MALA, "hmc": HMC, "nuts": NUTS, "aies": AIES, "aies_de": AIES_DE,
           "nuts_multinomial": NUTS_MULTINOMIAL}
LIK_EMULATOR, LIK_ANALYTIC = 0, 1
P_XI, P_ACCEPT, P_NUTS_DIR, P_NUTS_SEL, P_NUTS_TOP, P_AIES_PARTNER, P_AIES_Z = 1, 2, 3, 4, 5, 6, 7
P_INIT = 8  # initial walker positions
P_SWD = 9  # sliced-Wasserstein projection directions
INIT_REPEATED, INIT_UNIFORM, INIT_GAUSSIAN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liborc.so (gcc, OpenMP, -O2) if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_SO)
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Model(C.Structure):
    _fields_ = [
        ("lik_kind", C.c_int), ("d", C.c_int),
        ("d_c", C.c_int), ("n_hidden", C.c_int), ("n_data", C.c_int), ("linear", C.c_int),
        ("A", C.c_void_p), ("B", C.c_void_p), ("c", C.c_void_p), ("N", C.c_void_p),
        ("data", C.c_void_p), ("sigma", C.c_double),
        ("depth", C.c_int), ("width", C.c_int), ("params", C.c_void_p),
        ("in_m", C.c_void_p), ("in_s", C.c_void_p), ("out_m", C.c_double), ("out_s", C.c_double),
        ("bf16", C.c_int),
        ("lower", C.c_void_p), ("upper", C.c_void_p), ("gauss", C.c_void_p),
        ("mu", C.c_void_p), ("L", C.c_void_p),
        ("out_log", C.c_int), ("out_floor", C.c_double),
        ("pen_w", C.c_void_p),
    ]


class _StepParams(C.Structure):
    _fields_ = [
        ("kernel", C.c_int), ("eps", C.c_double), ("n_leapfrog", C.c_int), ("n_steps", C.c_int),
        ("max_depth", C.c_int), ("aies_a", C.c_double), ("aies_walkers", C.c_int),
        ("seed", C.c_uint64), ("de_sigma", C.c_double),
    ]


class _Trace(C.Structure):
    _fields_ = [
        ("samples", C.c_void_p), ("trace_logalpha", C.c_void_p), ("trace_logu", C.c_void_p),
        ("trace_accept", C.c_void_p), ("trace_depth", C.c_void_p), ("trace_nleaf", C.c_void_p),
        ("trace_margin", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = os.environ.get("ORC_SO") or build()
            L = C.CDLL(so)
            vp, d, i, u32, u64 = C.c_void_p, C.c_double, C.c_int, C.c_uint32, C.c_uint64
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_uniform.argtypes = [u64, u32, u32, u32, u32]
            L.orc_uniform.restype = d
            L.orc_normals.argtypes = [u64, u32, u32, u32, i, vp]
            L.orc_bf16_round.argtypes = [d]
            L.orc_bf16_round.restype = d
            L.orc_fp16_round.argtypes = [d]
            L.orc_fp16_round.restype = d
            L.orc_loglike.argtypes = [vp, vp, vp]
            L.orc_loglike.restype = d
            L.orc_loglike_batch.argtypes = [vp, i, vp, vp, vp]
            L.orc_logpost_z.argtypes = [vp, vp, vp, vp]
            L.orc_logpost_z.restype = d
            L.orc_logpost_batch.argtypes = [vp, i, vp, vp, vp]
            L.orc_leapfrog.argtypes = [vp, vp, vp, vp, d, i]
            L.orc_leapfrog.restype = d
            L.orc_run.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_run.restype = i
            L.orc_pooled_cov.argtypes = [i, i, vp, vp, vp]
            L.orc_chan_merge.argtypes = [i, d, vp, vp, d, vp, vp]
            L.orc_cholesky_jitter.argtypes = [i, vp, d, vp, vp]
            L.orc_cholesky_jitter.restype = i
            L.orc_remap_z.argtypes = [i, i, vp, vp, vp, vp, vp]
            L.orc_train_loss_grad.argtypes = [i, i, i, vp, vp, vp, d, d, i, d, i, i, vp, vp, vp]
            L.orc_train_loss_grad.restype = d
            L.orc_adam.argtypes = [i, vp, vp, vp, vp, i, d, d, d, d]
            L.orc_ess.argtypes = [i, i, i, vp, vp]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed, chain, it, purpose, idx):
    return lib().orc_uniform(seed, chain, it, purpose, idx)


def normals(seed, chain, it, purpose, n):
    out = np.zeros(n)
    lib().orc_normals(seed, chain, it, purpose, n, _ptr(out))
    return out


def bf16_round(v):
    return lib().orc_bf16_round(float(v))


def fp16_round(v):
    return lib().orc_fp16_round(float(v))


# --------------------------------------------------------------------------- model
class Model:
    """Owns the numpy arrays behind an ``orc_model`` (keeps them alive)."""

    def __init__(self, d, *, lik="emulator", lower=None, upper=None, gauss=None, mu=None, L=None,
                 analytic=None, emulator=None, bf16=False, fp16=False, pen_w=None):
        self._keep = []
        s = _Model()
        s.d = d
        if lik == "analytic":
            a = analytic
            s.lik_kind = LIK_ANALYTIC
            s.d_c = int(a.get("d_c", d))
            A, B, c = _f64(a["A"]), _f64(a["B"]), _f64(a["c"])
            s.n_data, s.n_hidden = A.shape
            s.linear = int(a.get("linear", False))
            N = _f64(a["N"]) if a.get("N") is not None else None
            data = _f64(a["data"])
            self._keep += [A, B, c, N, data]
            s.A, s.B, s.c, s.N, s.data = _ptr(A), _ptr(B), _ptr(c), _ptr(N), _ptr(data)
            s.sigma = float(a["sigma"])
        else:
            e = emulator
            s.lik_kind = LIK_EMULATOR
            s.depth, s.width = int(e["depth"]), int(e["width"])
            P = _f64(e["params"])
            in_m, in_s = _f64(e["in_m"]), _f64(e["in_s"])
            self._keep += [P, in_m, in_s]
            s.params, s.in_m, s.in_s = _ptr(P), _ptr(in_m), _ptr(in_s)
            s.out_m, s.out_s = float(e["out_m"]), float(e["out_s"])
            s.out_log, s.out_floor = int(e.get("out_log", 0)), float(e.get("out_floor", 0.0))
            s.bf16 = 2 if fp16 else int(bool(bf16))
        lower = _f64(np.full(d, -np.inf) if lower is None else lower)
        upper = _f64(np.full(d, np.inf) if upper is None else upper)
        mu = _f64(np.zeros(d) if mu is None else mu)
        L = _f64(np.eye(d) if L is None else L)
        g = None if gauss is None else np.ascontiguousarray(gauss, dtype=np.int32)
        self._keep += [lower, upper, mu, L, g]
        s.lower, s.upper, s.mu, s.L, s.gauss = _ptr(lower), _ptr(upper), _ptr(mu), _ptr(L), _ptr(g)
        pw = None if pen_w is None else _f64(pen_w)
        self._keep.append(pw)
        s.pen_w = _ptr(pw)
        self.s = s
        self.d = d

    @property
    def ref(self):
        return C.byref(self.s)

    def loglike(self, x, grad=True):
        x = _f64(np.atleast_2d(x))
        n = x.shape[0]
        out = np.zeros(n)
        g = np.zeros_like(x) if grad else None
        lib().orc_loglike_batch(self.ref, n, _ptr(x), _ptr(out), _ptr(g))
        return (out, g) if grad else out

    def logpost(self, z, grad=True):
        z = _f64(np.atleast_2d(z))
        n = z.shape[0]
        out = np.zeros(n)
        g = np.zeros_like(z) if grad else None
        lib().orc_logpost_batch(self.ref, n, _ptr(z), _ptr(out), _ptr(g))
        return (out, g) if grad else out


def leapfrog(model: Model, z, q, g, eps, n):
    z = _f64(z).copy(); q = _f64(q).copy(); g = _f64(g).copy()
    lp = lib().orc_leapfrog(model.ref, _ptr(z), _ptr(q), _ptr(g), float(eps), int(n))
    return z, q, g, lp


def run(model: Model, kernel, z, *, eps, n_steps, seed, n_leapfrog=10, max_depth=8, aies_a=2.0,
        aies_walkers=64, de_sigma=0.1, iter0=None, lp=None, g=None, record=True, trace=False):
    """Run n_steps of a sampler on all chains from whitened positions z[n][d].  de_sigma: the
    standard deviation of eta in the differential-evolution move (not given in Sec. 2.3).

    Returns a dict with the final state, per-chain counters and (optionally) the
    x-space samples [n_steps][n][d] and per-step decision traces."""
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    z = _f64(z).copy()
    n, d = z.shape
    if lp is None or g is None:
        lp0, g0 = model.logpost(z)
        lp = lp0 if lp is None else lp
        g = g0 if g is None else g
    lp = _f64(lp).copy()
    g = _f64(g).copy()
    it = np.zeros(n, dtype=np.uint32) if iter0 is None else np.ascontiguousarray(iter0, dtype=np.uint32).copy()
    acc_stat = np.zeros(n)
    accepts = np.zeros(n, dtype=np.int64)
    evals = np.zeros(n, dtype=np.int64)
    div = np.zeros(n, dtype=np.int64)
    p = _StepParams(kernel=k, eps=eps, n_leapfrog=n_leapfrog, n_steps=n_steps, max_depth=max_depth,
                    aies_a=aies_a, aies_walkers=aies_walkers, seed=seed, de_sigma=de_sigma)
    samples = np.zeros((n_steps, n, d)) if record else None
    t = _Trace()
    out = {}
    if record:
        t.samples = _ptr(samples)
    if trace:
        la = np.zeros((n_steps, n)); lu = np.zeros((n_steps, n))
        ac = np.zeros((n_steps, n), dtype=np.int32); dp = np.zeros((n_steps, n), dtype=np.int32)
        nl = np.zeros((n_steps, n), dtype=np.int32)
        mg = np.full((n_steps, n), np.inf)
        t.trace_logalpha, t.trace_logu, t.trace_accept = _ptr(la), _ptr(lu), _ptr(ac)
        t.trace_depth, t.trace_nleaf, t.trace_margin = _ptr(dp), _ptr(nl), _ptr(mg)
        out.update(log_alpha=la, log_u=lu, accept=ac, depth=dp, nleaf=nl, margin=mg)
    rc = lib().orc_run(model.ref, C.byref(p), n, _ptr(z), _ptr(lp), _ptr(g), _ptr(it), _ptr(acc_stat),
                       _ptr(accepts), _ptr(evals), _ptr(div), C.byref(t))
    if rc != 0:
        raise ValueError("orc_run rejected its arguments")
    out.update(z=z, lp=lp, g=g, iter=it, accept_stat=acc_stat, accepts=accepts, evals=evals,
               divergences=div, samples=samples)
    return out


# --------------------------------------------------------------------------- adaptation
def pooled_cov(x):
    x = _f64(x)
    n, d = x.shape
    mean = np.zeros(d); cov = np.zeros((d, d))
    lib().orc_pooled_cov(n, d, _ptr(x), _ptr(mean), _ptr(cov))
    return mean, cov


def chan_merge(na, mean_a, M2_a, nb, mean_b, M2_b):
    mean_a = _f64(mean_a).copy(); M2_a = _f64(M2_a).copy()
    mean_b = _f64(mean_b); M2_b = _f64(M2_b)
    lib().orc_chan_merge(mean_a.size, float(na), _ptr(mean_a), _ptr(M2_a), float(nb), _ptr(mean_b), _ptr(M2_b))
    return na + nb, mean_a, M2_a


def cholesky_jitter(S, jitter0=1e-10):
    S = _f64(S)
    d = S.shape[0]
    L = np.zeros((d, d)); used = np.zeros(1)
    rc = lib().orc_cholesky_jitter(d, _ptr(S), jitter0, _ptr(L), _ptr(used))
    return rc, L, float(used[0])


def remap_z(mu_old, L_old, mu_new, L_new, z):
    z = _f64(z).copy()
    n, d = z.shape
    lib().orc_remap_z(d, n, _ptr(_f64(mu_old)), _ptr(_f64(L_old)), _ptr(_f64(mu_new)), _ptr(_f64(L_new)), _ptr(z))
    return z


# --------------------------------------------------------------------------- training
def train_loss_grad(d, depth, width, params, in_m, in_s, out_m, out_s, X, chi2, out_log=0, out_floor=0.0,
                    bf16=False):
    P = _f64(params); X = _f64(X); y = _f64(chi2)
    g = np.zeros_like(P)
    loss = lib().orc_train_loss_grad(d, depth, width, _ptr(P), _ptr(_f64(in_m)), _ptr(_f64(in_s)),
                                     float(out_m), float(out_s), int(out_log), float(out_floor), int(bool(bf16)),
                                     X.shape[0],
                                     _ptr(X), _ptr(y), _ptr(g))
    return loss, g


def adam(p, g, m1, m2, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    p = _f64(p).copy(); m1 = _f64(m1).copy(); m2 = _f64(m2).copy(); g = _f64(g)
    lib().orc_adam(p.size, _ptr(p), _ptr(g), _ptr(m1), _ptr(m2), int(t), lr, b1, b2, eps)
    return p, m1, m2


# --------------------------------------------------------------------------- diagnostics
def ess(samples):
    """samples[n_draws][n_chains][d] -> ESS per dimension."""
    S = _f64(samples)
    n, M, d = S.shape
    out = np.zeros(d)
    lib().orc_ess(n, M, d, _ptr(S), _ptr(out))
    return out


def r_minus_1(samples):
    """Multivariate Gelman-Rubin statistic R - 1 (paper Sec. 4.1, the two displayed equations
    there): B = covariance of the chain means (chains - 1 denominator), W = mean over chains of
    the chain covariances (draws - 1 denominator), D = diag(sqrt(B_ii)), B~ = D^-1 B D^-1,
    W~ = D^-1 W D^-1, R - 1 = max_i |lambda_i| over the eigenvalues of W~^-1 B~.
    samples[n_draws][n_chains][d]; NaN when some B_ii is zero (the statistic is undefined)."""
    S = _f64(samples)
    n, M, d = S.shape
    means = S.mean(axis=0)                                   # [M][d]
    dm = means - means.mean(axis=0)
    B = dm.T @ dm / (M - 1)
    Y = S - means[None, :, :]                                # centred per chain
    W = np.einsum("tci,tcj->ij", Y, Y) / ((n - 1) * M)
    dB = np.sqrt(np.diag(B))
    if np.any(dB == 0.0):
        return float("nan")
    Bt = B / np.outer(dB, dB)
    Wt = W / np.outer(dB, dB)
    lam = np.linalg.eigvals(np.linalg.solve(Wt, Bt))
    return float(np.max(np.abs(lam)))


def draw_positions(strategy, seed, n, d, *, center=None, Lc=None, lower=None, upper=None):
    """Initial walker positions (the initialisation strategies of Sec. 3.1): REPEATED every
    chain at `center`; UNIFORM lower + (upper - lower) u with u the uniforms 0..d-1 of stream
    (chain, 0, P_INIT); GAUSSIAN center + Lc xi with xi the normals 0..d-1 of that stream.
    Returns theta[n][d]."""
    out = np.zeros((n, d))
    for c in range(n):
        if strategy == INIT_REPEATED:
            out[c] = _f64(center)
        elif strategy == INIT_UNIFORM:
            u = np.array([uniform(seed, c, 0, P_INIT, i) for i in range(d)])
            out[c] = _f64(lower) + (_f64(upper) - _f64(lower)) * u
        elif strategy == INIT_GAUSSIAN:
            out[c] = _f64(center) + _f64(Lc) @ normals(seed, c, 0, P_INIT, d)
        else:
            raise ValueError("unknown strategy")
    return out


def w1_1d(a, b):
    """1-D Wasserstein-1 distance of two empirical distributions: the integral over t in (0, 1)
    of |F^-1(t) - G^-1(t)|.  With na, nb values the quantile functions step at multiples of
    1/na and 1/nb; over the common denominator na nb the breakpoints are the integers T = i nb
    and j na, and on the interval ending at T the quantile functions take the sorted values of
    ranks ceil(T / nb) - 1 and ceil(T / na) - 1 (integer arithmetic: exact interval ends)."""
    a = np.sort(_f64(a).ravel())
    b = np.sort(_f64(b).ravel())
    na, nb = len(a), len(b)
    T = np.union1d(np.arange(1, na + 1, dtype=np.int64) * nb, np.arange(1, nb + 1, dtype=np.int64) * na)
    ia = (T + nb - 1) // nb - 1
    ib = (T + na - 1) // na - 1
    width = np.diff(np.concatenate(([0], T))) / (float(na) * float(nb))
    return float(np.sum(width * np.abs(a[ia] - b[ib])))


def swd_directions(seed, n_proj, d):
    """Projection directions of the sliced Wasserstein distance: direction k is the normals
    0..d-1 of stream (k, 0, P_SWD), normalised (uniform on the sphere); the same set is reused
    for every comparison, as in Sec. 4.1."""
    u = np.array([normals(seed, k, 0, P_SWD, d) for k in range(n_proj)])
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def sliced_wasserstein(P, Q, *, n_proj=500, seed=0):
    """Sliced Wasserstein distance (Sec. 4.1): the mean over the projection directions u_k of
    the 1-D Wasserstein-1 distance between the projections P u_k and Q u_k (P[n][d], Q[m][d])."""
    P = _f64(P).reshape(-1, np.shape(P)[-1])
    Q = _f64(Q).reshape(-1, np.shape(Q)[-1])
    U = swd_directions(seed, n_proj, P.shape[1])
    return float(np.mean([w1_1d(P @ u, Q @ u) for u in U]))


def quantiles(samples, q):
    """Per-dimension quantiles of the pooled draws samples[n_draws][n_chains][d] at levels q
    (linear interpolation between order statistics at rank (N - 1) q); out[d][len(q)]."""
    S = _f64(samples)
    flat = S.reshape(-1, S.shape[-1])
    return np.quantile(flat, np.asarray(q, dtype=np.float64), axis=0).T.copy()


def credible_metric(samples, alpha, true_lo, true_hi):
    """Credible metric of Sec. 4.1 per dimension: (|hi - hi0| + |lo - lo0|) / (hi0 - lo0), with
    lo, hi the equal-tailed credible limits at level alpha of the pooled draws (quantiles
    (1 - alpha) / 2 and (1 + alpha) / 2) and lo0, hi0 the true limits."""
    lo0 = _f64(true_lo)
    hi0 = _f64(true_hi)
    qs = quantiles(samples, [(1.0 - alpha) / 2.0, (1.0 + alpha) / 2.0])
    return (np.abs(qs[:, 1] - hi0) + np.abs(qs[:, 0] - lo0)) / (hi0 - lo0)


def n_params(d, depth, width):
    return d * width + width + (depth - 1) * (width * width + width) + width + 1
