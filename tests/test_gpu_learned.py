"""The learned part: an emulator trained on the GPU by the library's own forward,
backward and Adam kernels, on (theta, chi^2) pairs labelled by the plain
method's FP64 analytic likelihood; the analytic likelihood measures its error
along sampled chains."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def test_training_reduces_emulator_error_along_chains():
    from paper_2606_04895_gb300 import Sampler
    from paper_2606_04895_gb300 import learn
    tgt = S.target(6, seed=0)
    emu, hist, (in_m, in_s, out_m, out_s) = learn.train_emulator(
        tgt, n_train=1 << 16, width=256, depth=3, epochs=12, batch=2048, lr=2e-3, precision="fp32", n_chains=256)
    assert hist["train_loss"][-1] < 0.2 * hist["train_loss"][0]
    assert hist["val_mse"][-1] < 0.1
    # chains of the plain method around the posterior
    plain = learn.analytic_sampler(tgt, n_chains=256, precision="fp32", seed=3)
    Lp = np.linalg.cholesky(tgt["laplace_cov"])
    th0 = tgt["theta_star"] + S.chains_init(256, 6, seed=5) @ Lp.T
    plain.init_chains(th0, tgt["lower"], tgt["upper"], mu=tgt["theta_star"], L=Lp)
    out = torch.empty((200, 256, 6), dtype=torch.float32, device="cuda")
    plain.step("mala", 200, eps=0.4, samples=out)
    truth = learn.analytic_sampler(tgt, n_chains=1, precision="fp64")
    err_trained = learn.dlogl_along_chains(emu, truth, out).cpu().numpy()
    # the same network before training
    e0 = S.emulator(6, width=256, depth=3, seed=5, in_m=in_m, in_s=in_s, out_m=out_m, out_s=out_s)
    raw = Sampler(6, 8, precision="fp32", likelihood="emulator")
    raw.set_emulator(e0["params"], 3, 256, in_m, in_s, out_m, out_s)
    err_raw = learn.dlogl_along_chains(raw, truth, out).cpu().numpy()
    print(f"|dlogL| along chains: trained median {np.median(err_trained):.3g}, untrained {np.median(err_raw):.3g}")
    assert np.median(err_trained) < 0.1 * np.median(err_raw)
    for s in (emu, plain, truth, raw):
        s.close()
