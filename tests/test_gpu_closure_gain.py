"""What the trained learned closure gains over the method without it.

A fine run (FP32 path, 4x finer than the coarse grid, moist layer with a
k^-5/3 random-phase velocity field reaching the coarse subgrid scales) is
top-hat filtered onto the coarse nodes by the library's filter kernel; the
closure network is trained on one such run with the library's BF16
tensor-core forward/backward kernels and Adam, and evaluated on a second run with
different random phases against the filtered subgrid targets, next to
Smagorinsky-Lilly (C_s = 0.21 with the Richardson correction) evaluated on the
same filtered gradients and each sample's filtered theta_v.  A priori test: the error measure is the relative L2
distance of the predicted eddy viscosity / diffusivity from the least-squares
targets nu*, kappa*.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sl(X, thv, Cs=0.21, Prt=1.0 / 3.0, g=9.81):
    """Smagorinsky-Lilly with the Richardson correction (Eqs. smago,
    richardson) on the filtered gradients of each sample, with the sample's
    own filtered theta_v in the Richardson number."""
    gu = X[:, :9].reshape(-1, 3, 3)
    S = 0.5 * (gu + gu.transpose(0, 2, 1))
    S2 = 2.0 * (S ** 2).sum(axis=(1, 2))
    Smag = np.sqrt(S2)
    Ri = np.where(S2 > 0, g / thv * X[:, 11] / np.maximum(S2, 1e-300), 0.0)
    fb = np.where(Ri <= 0, 1.0, np.maximum(0.0, 1.0 - Ri / Prt) ** 0.25)
    nu = (Cs * X[:, 12]) ** 2 * Smag * fb
    return nu, nu / Prt


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_trained_closure_beats_smagorinsky_a_priori():
    from paper_2110_00853_b300 import closure
    sub = (64, 64, 32)
    Xtr, Ttr = closure.fine_run_samples(torch, steps=20, seed=4, sub=sub)
    Xte, Tte, thv_te = closure.fine_run_samples(torch, steps=20, seed=44, sub=sub, with_thv=True)
    assert Xtr.shape[0] == 16 * 16 * 8 * 125
    assert bool(torch.isfinite(Xtr).all()) and bool(torch.isfinite(Ttr).all())
    P, hist = closure.fit(torch, Xtr, Ttr, steps=1500, batch=65536, lr=2e-3, log_every=100)
    nu_m, ka_m = (a.cpu().numpy().astype(np.float64) for a in closure.predict(torch, P, Xte))
    x = Xte.cpu().numpy().astype(np.float64)
    t = Tte.cpu().numpy().astype(np.float64)
    nu_sl, ka_sl = _sl(x, thv_te.cpu().numpy().astype(np.float64))
    e = dict(nu_mlp=_rel(nu_m, t[:, 0]), nu_sl=_rel(nu_sl, t[:, 0]), ka_mlp=_rel(ka_m, t[:, 1]),
             ka_sl=_rel(ka_sl, t[:, 1]))
    print("loss history", hist)
    print("a priori relative L2 errors on held-out samples", e)
    assert hist[-1] < hist[0]
    assert e["nu_mlp"] < e["nu_sl"] and e["ka_mlp"] < e["ka_sl"]
