"""Learned SGS closure: training-data generation and GPU training loop.

Orchestration only.  The fine-resolution run, the box filter that turns it
into (input, target) samples, the network's forward and backward passes and
the Adam update all run in the library's CUDA kernels (cmles_step,
cmles_closure_samples, cmles_mlp_loss_grad, cmles_mlp_adam); this module
chooses the batches and the normalisation constants.

The paper has no learned closure.  This extension of its Sec. 4 is a network
13 -> 64 -> 64 -> 2 trained on box-filtered fine-resolution runs, with
Smagorinsky-Lilly kept as the fallback and as the yardstick of its error.
"""
import math

import numpy as np

from . import cmles
from . import inputs as I


def init_params(seed=0, in_scale=None, out_scale=(1.0, 1.0), b3=(0.0, 0.0)):
    """Seeded initial parameter vector (FP32, 5201 values): scaled normal
    weights (variance 1/fan_in), zero hidden biases, given output biases and
    normalisation constants."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(size=(64, 13)) / math.sqrt(13), np.zeros(64),
             rng.normal(size=(64, 64)) / math.sqrt(64), np.zeros(64),
             rng.normal(size=(2, 64)) / math.sqrt(64) * 0.1, np.asarray(b3, float),
             np.ones(13) if in_scale is None else np.asarray(in_scale, float), np.asarray(out_scale, float)]
    return np.concatenate([np.ravel(p) for p in parts]).astype(np.float32)


def fine_run_samples(torch, name="c4fine", steps=20, dt=0.005, factor=4, nmodes=2000, kmax=200, seed=4,
                     sub=None, with_thv=False):
    """Run the fine mesh (FP32 path, Smagorinsky-Lilly) from a state with a
    k^-5/3 random-phase velocity field that reaches the subgrid scales of the
    coarse mesh, then filter it onto the coarse nodes: (X, T), and the
    filtered theta_v with with_thv."""
    mesh = I.mesh(name) if sub is None else I.sub_mesh(name, *sub)
    phys = I.physics(name)
    phys["dt"] = dt
    case = I.case(name)
    case["modes"] = I.velocity_modes(mesh["Lx"], mesh["Ly"], mesh["Lz"], nmodes=nmodes, kmax=kmax, seed=seed)
    G = cmles.Solver(mesh, phys, precision="fp32")
    G.init_case(case)
    G.step(steps)
    out = G.closure_samples(factor, with_thv=with_thv)
    G.close()
    return out


def normalisation(X, T):
    """in_scale = 1/std of each input (Delta: 1/mean), out_scale = std of the
    targets; computed on the host from a copy of the samples."""
    x = X.cpu().numpy().astype(np.float64)
    t = T.cpu().numpy().astype(np.float64)
    in_scale = 1.0 / np.maximum(x.std(axis=0), 1e-30)
    in_scale[12] = 1.0 / max(abs(x[:, 12].mean()), 1e-30)
    out_scale = np.maximum(t.std(axis=0), 1e-30)
    return in_scale, out_scale


def fit(torch, X, T, steps=2000, batch=65536, lr=2e-3, seed=0, log_every=0):
    """Train the closure network on samples (X raw features, T raw targets):
    returns the FP32 parameter vector (device tensor) including the
    normalisation constants, and the loss history."""
    in_scale, out_scale = normalisation(X, T)
    p = init_params(seed, in_scale, out_scale)
    P = torch.from_numpy(p).cuda()
    Xs = (X * torch.from_numpy(in_scale.astype(np.float32)).cuda()).contiguous()
    Ts = (T / torch.from_numpy(out_scale.astype(np.float32)).cuda()).contiguous()
    M = torch.zeros(cmles.MLP_NET, device="cuda")
    V = torch.zeros(cmles.MLP_NET, device="cuda")
    n = X.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    hist = []
    for t in range(1, steps + 1):
        idx = torch.randint(0, n, (min(batch, n),), device="cuda", generator=g)
        loss, grad = cmles.mlp_loss_grad(P, Xs[idx].contiguous(), Ts[idx].contiguous())
        cmles.mlp_adam(P, grad, M, V, t, lr=lr)
        if log_every and t % log_every == 0:
            hist.append(float(loss.item()))
    return P, hist


def predict(torch, P, X):
    """(nu_t, D_t) of the closure for raw features X, as the DG kernels
    evaluate it: nu = out_scale0 max(y0, 0), D = out_scale1 max(y1, 0)."""
    p = P.cpu().numpy()
    in_scale = torch.from_numpy(p[cmles.MLP_NET:cmles.MLP_NET + 13].copy()).cuda()
    out_scale = p[cmles.MLP_NET + 13:]
    Y = cmles.mlp_forward(P, (X * in_scale).contiguous())
    return (torch.clamp(Y[:, 0], min=0.0) * float(out_scale[0]), torch.clamp(Y[:, 1], min=0.0) * float(out_scale[1]))
