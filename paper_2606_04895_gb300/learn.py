"""Training the likelihood emulator on data the plain method generates.

The plain method is the analytic "theory map" likelihood; its FP64 GPU path
labels each training input with chi^2 = -2 logL.  The emulator (tanh MLP,
paper Sec. 1 and Sec. 4: a neural-network likelihood that replaces the
parameter-to-likelihood pipeline) is then fitted with the library's own
forward / backward / Adam kernels (bst_train_step): MSE on the standardised
chi^2, Adam (Kingma & Ba) on FP32 master weights, batches of 4096.  The
analytic likelihood stays available to measure the emulator's error
along sampled chains.

Only argument marshalling and batching happen here; every evaluation,
gradient and optimiser update runs in libbst's CUDA kernels.  The
standardisation constants (mean / sd of the inputs and of the labels) are
computed once from the host copy of the training set.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Sampler


def analytic_sampler(tgt, n_chains=1, precision="fp64", seed=0):
    """A library handle on the analytic likelihood of a synthetic target dict."""
    s = Sampler(tgt["d"], n_chains, precision=precision, likelihood="analytic", seed=seed)
    s.set_analytic(tgt["A"], tgt["B"], tgt["c"], tgt["data"], tgt["sigma"], d_c=tgt["d_c"], N=tgt["N"],
                   linear=tgt["linear"])
    return s


def label(plain: Sampler, theta: np.ndarray, chunk=1 << 18) -> np.ndarray:
    """chi^2 = -2 logL of the plain (analytic) likelihood at every row of theta (GPU, FP64)."""
    out = np.empty(len(theta))
    for i in range(0, len(theta), chunk):
        x = torch.as_tensor(theta[i:i + chunk], dtype=torch.float64, device=plain.device)
        out[i:i + chunk] = -2.0 * plain.loglike(x).cpu().numpy()
    return out


def standardisation(theta: np.ndarray, chi2: np.ndarray):
    return theta.mean(axis=0), theta.std(axis=0) + 1e-12, float(chi2.mean()), float(chi2.std() + 1e-12)


def log_output_standardisation(chi2: np.ndarray, margin=1.0):
    """Log output transform: floor = min(chi2) - margin, then the mean / sd of log(chi2 - floor)
    (the regression target of the log output, bst_set_emulator_output)."""
    floor = float(chi2.min() - margin)
    y = np.log(chi2 - floor)
    return floor, float(y.mean()), float(y.std() + 1e-12)


def fit(emu: Sampler, theta: np.ndarray, chi2: np.ndarray, *, epochs=4, batch=4096, lr=1e-3, lr_min=None, seed=0,
        val_frac=1 / 64, log=None):
    """Adam on the emulator held by `emu` (its set_emulator weights are the start); with lr_min
    the step size follows a cosine from lr to lr_min over the epochs.

    Returns a dict with the per-epoch training loss and validation MSE (on the
    standardised regression target)."""
    n = len(theta)
    n_val = max(1, int(n * val_frac))
    X = torch.as_tensor(theta, dtype=torch.float32, device=emu.device)
    Y = torch.as_tensor(chi2, dtype=torch.float32, device=emu.device)
    Xv, Yv = X[:n_val], Y[:n_val]
    Xt, Yt = X[n_val:], Y[n_val:]
    g = torch.Generator(device=emu.device)
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=emu.device)
    hist = {"train_loss": [], "val_mse": []}
    nt = len(Xt)
    for ep in range(epochs):
        lr_ep = lr if lr_min is None else lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * ep / max(epochs, 1)))
        perm = torch.randperm(nt, device=emu.device, generator=g)
        acc = torch.zeros(1, dtype=torch.float32, device=emu.device)
        nb = 0
        for i in range(0, nt - batch + 1, batch):
            idx = perm[i:i + batch]
            emu.train_step(Xt.index_select(0, idx), Yt.index_select(0, idx), lr=lr_ep, loss_out=loss)
            acc += loss
            nb += 1
        vl, _ = emu.train_grad(Xv, Yv)
        hist["train_loss"].append(float(acc.item() / max(nb, 1)))
        hist["val_mse"].append(float(vl.item()))
        if log:
            log(f"epoch {ep + 1}: train {hist['train_loss'][-1]:.4g} val {hist['val_mse'][-1]:.4g}")
    return hist


def train_emulator(tgt, *, n_train=1 << 20, width=512, depth=4, epochs=4, batch=4096, lr=1e-3, seed=4,
                   precision="bf16", n_chains=4096, log=None):
    """Config-4 recipe: 50 % box-uniform / 50 % Gaussian-at-3-sigma inputs, FP64 analytic
    labels, MSE on the standardised chi^2.  Returns (sampler with the trained emulator,
    training history, standardisation)."""
    import synthetic as S
    theta = S.training_inputs(tgt, n_train, seed=seed)
    plain = analytic_sampler(tgt)
    chi2 = label(plain, theta)
    plain.close()
    in_m, in_s, out_m, out_s = standardisation(theta, chi2)
    e = S.emulator(tgt["d"], width=width, depth=depth, seed=seed + 1, in_m=in_m, in_s=in_s, out_m=out_m,
                   out_s=out_s)
    emu = Sampler(tgt["d"], n_chains, precision=precision, likelihood="emulator", seed=seed)
    emu.set_emulator(e["params"], depth, width, in_m, in_s, out_m, out_s)
    hist = fit(emu, theta, chi2, epochs=epochs, batch=batch, lr=lr, seed=seed, log=log)
    return emu, hist, (in_m, in_s, out_m, out_s)


def input_whitening(tgt, scale2=9.0):
    """Centre and whitening matrix of the emulator's input: u = T (theta - c) with c = theta* and
    T = chol(scale2 Sigma_Laplace)^-1, the Gaussian half of the training inputs mapped to N(0, I)
    (the posterior core at unit scale).  Returns (c, T)."""
    c = np.asarray(tgt["theta_star"], dtype=np.float64)
    T = np.linalg.inv(np.linalg.cholesky(scale2 * np.asarray(tgt["laplace_cov"], dtype=np.float64)))
    return c, T


def fold_input_map(e, c, T):
    """The emulator with its input map u = T (x - c) folded into layer 1 (W_1 <- W_1 T,
    b_1 <- b_1 - W_1 T c) and identity standardisation; the network function is unchanged."""
    import synthetic as S
    W, b, wo, bo = S.unpack_emulator(e)
    W1 = W[0] @ T
    W = [W1] + list(W[1:])
    b = [b[0] - W1 @ c] + list(b[1:])
    return dict(e, params=S.pack_emulator(W, b, wo, bo), in_m=np.zeros(len(c)), in_s=np.ones(len(c)))


def train_emulator_log(tgt, *, n_train=1 << 20, width=512, depth=4, epochs=40, batch=4096, lr=1e-3, lr_min=1e-5,
                       seed=4, log=None, device=None, precision="bf16", gauss_frac=0.5, gauss_scale=3.0):
    """Config-4 recipe with the log output and whitened inputs: 50 % box-uniform / 50 %
    Gaussian-at-3-sigma inputs (2^20; `gauss_frac` and `gauss_scale` set the Gaussian share and
    its widths, and the input whitening maps the first width to N(0, I)), FP64 analytic
    chi^2 labels, MSE on the standardised log(chi2 - floor), Adam (lr 1e-3, cosine to lr_min) on
    FP32 masters in batches of 4096, all in the library's training kernels: precision "bf16"
    trains the hidden layers on the tensor cores (BF16 operands, FP32 accumulation), "fp32" on
    the CUDA cores.  The input is
    u = T (theta - theta*) (input_whitening), folded into layer 1 afterwards.  Returns (emulator
    dict with the trained weights, history, the training inputs and labels)."""
    import synthetic as S
    d = tgt["d"]
    theta = S.training_inputs(tgt, n_train, seed=seed, gauss_frac=gauss_frac, gauss_scale=gauss_scale)
    plain = analytic_sampler(tgt)
    chi2 = label(plain, theta)
    plain.close()
    s0 = gauss_scale if np.isscalar(gauss_scale) else gauss_scale[0]
    c, T = input_whitening(tgt, scale2=s0 ** 2)
    u = (theta - c) @ T.T
    floor, out_m, out_s = log_output_standardisation(chi2)
    e0 = S.emulator(d, width=width, depth=depth, seed=seed + 1, in_m=np.zeros(d), in_s=np.ones(d), out_m=out_m,
                    out_s=out_s, out_log=1, out_floor=floor)
    emu = Sampler(d, 8, precision=precision, likelihood="emulator", seed=seed,
                  **({} if device is None else {"device": device}))
    emu.set_emulator(e0["params"], depth, width, e0["in_m"], e0["in_s"], out_m, out_s, out_log=1, out_floor=floor)
    hist = fit(emu, u, chi2, epochs=epochs, batch=batch, lr=lr, lr_min=lr_min, seed=seed, log=log)
    e = fold_input_map(dict(e0, params=emu.get_emulator()), c, T)
    emu.close()
    return e, hist, (theta, chi2)


def emulator_sampler(e, n_chains, precision="bf16", seed=0, device=None):
    """A library handle on the emulator dict `e` (weights, standardisation, output transform)."""
    s = Sampler(e["d"], n_chains, precision=precision, likelihood="emulator", seed=seed,
                **({} if device is None else {"device": device}))
    s.set_emulator(e["params"], e["depth"], e["width"], e["in_m"], e["in_s"], e["out_m"], e["out_s"],
                   out_log=e.get("out_log", 0), out_floor=e.get("out_floor", 0.0))
    return s


def dlogl_along_chains(emu: Sampler, plain: Sampler, samples: torch.Tensor):
    """|logL_emulator - logL_plain| at sampled points (x-space rows of `samples`)."""
    x = samples.reshape(-1, samples.shape[-1])
    le = emu.loglike(x.to(emu.dtype)).double()
    lp = plain.loglike(x.to(plain.dtype)).double()
    return (le - lp).abs()
