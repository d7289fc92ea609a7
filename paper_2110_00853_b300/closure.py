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


def normalisation(X, T, max_rows=4_000_000):
    """in_scale = 1/std of each input (Delta: 1/mean), out_scale = std of the
    targets; computed on the host from a copy of the samples (every k-th one
    when there are more than max_rows)."""
    k = max(1, -(-X.shape[0] // max_rows))
    x = X[::k].cpu().numpy().astype(np.float64)
    t = T[::k].cpu().numpy().astype(np.float64)
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


# ---------------------------------------------------------------------------
# The learned-closure configuration at its stated scale: training data from
# the 128 x 128 x 64-element fine mesh (131M nodes, FP32) box-filtered 4x onto
# the 32 x 32 x 16-element coarse mesh, about 2e8 samples; then the coarse
# runs with the trained closure and with Smagorinsky-Lilly judged a
# posteriori against a fine run from the same initial state, on the
# kinetic-energy spectrum and the horizontal-mean theta and q_t profiles.

def _levels_z(m):
    """heights of the node levels (ez, k) of a flat N = 4 mesh, bottom to top
    (the LGL nodes 0, +-sqrt(3/7), +-1)"""
    assert m["N"] == 4
    xi = np.array([-1.0, -math.sqrt(3.0 / 7.0), 0.0, math.sqrt(3.0 / 7.0), 1.0])
    hz = m["Lz"] / m["nez"]
    return np.array([m["z0"] + (ez + 0.5 * (x + 1.0)) * hz for ez in range(m["nez"]) for x in xi])


def c4_experiment(torch, train_seeds=(4, 5, 6, 7, 8), test_seed=44, steps=2000, snap_every=100, dt_fine=0.005,
                  dt_coarse=0.02, fit_steps=6000, kmax_train=200, kmax_test=32, nshell_cmp=48, log=print):
    """Runs the configuration and returns its figures (a dict)."""
    import time
    out = dict(config=dict(fine="c4fine 128x128x64", coarse="c2 32x32x16", steps=steps, snap_every=snap_every,
                           dt_fine=dt_fine, dt_coarse=dt_coarse, fit_steps=fit_steps, kmax_train=kmax_train,
                           kmax_test=kmax_test, train_seeds=list(train_seeds), test_seed=test_seed))
    mf, mc = I.mesh("c4fine"), I.mesh("c2")
    pf = dict(I.physics("c4fine"), dt=dt_fine)
    # 1. training samples: fine runs from random-phase fields reaching the
    #    coarse subgrid scales, filtered every snap_every steps
    Xs, Ts = [], []
    t0 = time.time()
    for seed in train_seeds:
        case = I.case("c4fine")
        case["modes"] = I.velocity_modes(mf["Lx"], mf["Ly"], mf["Lz"], nmodes=2000, kmax=kmax_train, seed=seed)
        G = cmles.Solver(mf, pf, precision="fp32")
        G.init_case(case)
        for k in range(steps // snap_every):
            G.step(snap_every)
            X, T = G.closure_samples(4)
            Xs.append(X)
            Ts.append(T)
        d = G.diagnostics()
        assert not d["nonfinite"]
        G.close()
        log(f"fine training run seed {seed}: {len(Xs)} snapshots, {time.time() - t0:.0f} s")
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    del Xs, Ts
    out["samples"] = int(X.shape[0])
    out["fine_train_seconds"] = time.time() - t0
    # 2. training on the GPU (forward / backward on the tensor cores, Adam)
    t0 = time.time()
    P, hist = fit(torch, X, T, steps=fit_steps, batch=65536, lr=2e-3, log_every=max(fit_steps // 20, 1))
    torch.cuda.synchronize()
    out["fit_seconds"] = time.time() - t0
    out["loss_history"] = hist
    del X, T
    torch.cuda.empty_cache()
    log(f"trained on {out['samples']} samples: loss {hist[0]:.4g} -> {hist[-1]:.4g}")
    # 3. the test: one initial state (random phases, resolved on the coarse mesh)
    def case_test(m):
        c = I.case("c2")
        c["modes"] = I.velocity_modes(m["Lx"], m["Ly"], m["Lz"], nmodes=1000, kmax=kmax_test, seed=test_seed)
        return c
    tend = steps * dt_fine
    G = cmles.Solver(mf, pf, precision="fp32")
    G.init_case(case_test(mf))
    E0f = G.spectrum(nshell_cmp + 1)
    t0 = time.time()
    G.step(int(round(tend / dt_fine)))
    out["fine_test_seconds"] = time.time() - t0
    Ef = G.spectrum(nshell_cmp + 1)
    prof_f = G.profiles()
    G.close()
    zf = _levels_z(mf)
    zc = _levels_z(mc)
    th_f = np.interp(zc, zf, prof_f[:, 1])
    qt_f = np.interp(zc, zf, prof_f[:, 2])
    runs = {}
    for name, prec, clo in (("learned_fp32", "fp32", "mlp"), ("sl_fp32", "fp32", "sl"), ("sl_fp64", "fp64", "sl")):
        pc = dict(I.physics("c2", closure=clo), dt=dt_coarse)
        G = cmles.Solver(mc, pc, precision=prec)
        G.init_case(case_test(mc))
        if clo == "mlp":
            G.set_closure_weights_device(P)
        E0c = G.spectrum(nshell_cmp + 1)
        G.step(int(round(tend / dt_coarse)))
        Ec = G.spectrum(nshell_cmp + 1)
        pr = G.profiles()
        d = G.diagnostics(raise_on_error=False)
        G.close()
        sl = slice(1, nshell_cmp + 1)
        lo = slice(1, nshell_cmp // 2 + 1)
        runs[name] = dict(
            spectrum_rel_l2_low=float(np.linalg.norm(Ec[lo] - Ef[lo]) / np.linalg.norm(Ef[lo])),
            spectrum_log_rms_low=float(np.sqrt(np.mean(np.log(np.maximum(Ec[lo], 1e-300) / Ef[lo]) ** 2))),
            finite=not d["nonfinite"],
            spectrum_rel_l2=float(np.linalg.norm(Ec[sl] - Ef[sl]) / np.linalg.norm(Ef[sl])),
            spectrum_log_rms=float(np.sqrt(np.mean(np.log(np.maximum(Ec[sl], 1e-300) / Ef[sl]) ** 2))),
            ke_rel=float(abs(Ec[sl].sum() - Ef[sl].sum()) / Ef[sl].sum()),
            theta_max_abs=float(np.abs(pr[:, 1] - th_f).max()),
            qt_max_abs=float(np.abs(pr[:, 2] - qt_f).max()),
            initial_spectrum_rel_l2=float(np.linalg.norm(E0c[sl] - E0f[sl]) / np.linalg.norm(E0f[sl])),
            spectrum=Ec.tolist())
        log(name, {k: v for k, v in runs[name].items() if k != "spectrum"})
    out["runs"] = runs
    out["fine_spectrum"] = Ef.tolist()
    out["fine_initial_spectrum"] = E0f.tolist()
    out["t_end_s"] = tend
    return out


if __name__ == "__main__":
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser(description="learned-closure configuration at its stated scale")
    ap.add_argument("--out", required=True, help="JSON file of the figures")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--fit-steps", type=int, default=6000)
    ap.add_argument("--seeds", default="4,5,6,7,8")
    a = ap.parse_args()
    res = c4_experiment(torch, train_seeds=tuple(int(s) for s in a.seeds.split(",")), steps=a.steps,
                        fit_steps=a.fit_steps)
    with open(a.out, "w") as f:
        json.dump(res, f)
