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


def fit(emu: Sampler, theta: np.ndarray, chi2: np.ndarray, *, epochs=4, batch=4096, lr=1e-3, seed=0,
        val_frac=1 / 64, log=None):
    """Adam on the emulator held by `emu` (its set_emulator weights are the start).

    Returns a dict with the per-epoch training loss and validation MSE (on the
    standardised chi^2)."""
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
        perm = torch.randperm(nt, device=emu.device, generator=g)
        acc = torch.zeros(1, dtype=torch.float32, device=emu.device)
        nb = 0
        for i in range(0, nt - batch + 1, batch):
            idx = perm[i:i + batch]
            emu.train_step(Xt.index_select(0, idx), Yt.index_select(0, idx), lr=lr, loss_out=loss)
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


def dlogl_along_chains(emu: Sampler, plain: Sampler, samples: torch.Tensor):
    """|logL_emulator - logL_plain| at sampled points (x-space rows of `samples`)."""
    x = samples.reshape(-1, samples.shape[-1])
    le = emu.loglike(x.to(emu.dtype)).double()
    lp = plain.loglike(x.to(plain.dtype)).double()
    return (le - lp).abs()
