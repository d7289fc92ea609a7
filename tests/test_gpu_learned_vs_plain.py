"""The FP32 path with the trained learned closure against the plain FP64
method with Smagorinsky-Lilly, a posteriori: the same moist-layer box
(16 x 16 x 8 elements of the moist-layer grid, 200 m elements) started from a
k^-5/3 random-phase velocity field is run 500 steps (10 s) both ways, and the
resolved kinetic energy and the horizontal-mean theta and q_t profiles
(Favre means, App. C) are compared.  A third run, FP32 with Smagorinsky-
Lilly, separates the precision's share of the difference from the
closure's.  The closure is trained as in the a priori test (fine run box-
filtered 4x, GPU forward/backward kernels, Adam)."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ke(Q, wq, J):
    rho = Q[:, 0]
    m2 = (Q[:, 1:4] ** 2).sum(1)
    return float((0.5 * m2 / rho * wq[None, :]).sum() * J)


def test_learned_fp32_against_plain_fp64(orc):
    from paper_2110_00853_b300 import closure, cmles
    Xtr, Ttr = closure.fine_run_samples(torch, steps=20, seed=4, sub=(64, 64, 32))
    P, _ = closure.fit(torch, Xtr, Ttr, steps=1500, batch=65536, lr=2e-3)
    del Xtr, Ttr
    m = I.sub_mesh("c2", 16, 16, 8)
    case = I.case("c2")
    case["modes"] = I.velocity_modes(m["Lx"], m["Ly"], m["Lz"], nmodes=500, kmax=24, seed=7)
    _, w, _ = orc.lgl(4)
    wq = torch.tensor(np.einsum("k,j,i->kji", w, w, w).ravel(), device="cuda", dtype=torch.float64)
    J = (m["Lx"] / m["nex"]) * (m["Ly"] / m["ney"]) * (m["Lz"] / m["nez"]) / 8.0
    out = {}
    for name, prec, clo in (("plain64", "fp64", "sl"), ("plain32", "fp32", "sl"), ("learned32", "fp32", "mlp")):
        G = cmles.Solver(m, I.physics("c2", closure=clo), precision=prec)
        G.init_case(case)
        if clo == "mlp":
            G.set_closure_weights_device(P)
        ke0 = _ke(G.get_state(), wq, J)
        G.step(500)
        Q = G.get_state()
        d = G.diagnostics()
        prof = G.profiles()
        out[name] = dict(ke0=ke0, ke=_ke(Q, wq, J), theta=prof[:, 1], qt=prof[:, 2])
        G.close()
    p = out["plain64"]
    print("resolved KE: initial", p["ke0"], "after 10 s", {k: v["ke"] for k, v in out.items()})
    for k in ("plain32", "learned32"):
        dke = abs(out[k]["ke"] - p["ke"]) / p["ke"]
        dth = np.abs(out[k]["theta"] - p["theta"]).max()
        dq = np.abs(out[k]["qt"] - p["qt"]).max()
        out[k].update(dke=dke, dth=dth, dq=dq)
        print(k, "vs plain FP64: KE rel", dke, "theta max |d| K", dth, "q_t max |d|", dq)
    # measured: FP32 + SL 3.3e-7 in KE, 1.6e-6 K in theta; FP32 + learned
    # 7.8e-4 in KE, 2.9e-3 K in theta, 1.6e-5 in q_t (the closure's different
    # dissipation).  Bounds about 5x the measurements.
    assert out["plain32"]["dke"] < 2e-6 and out["plain32"]["dth"] < 1e-5
    assert out["learned32"]["dke"] < 5e-3 and out["learned32"]["dth"] < 2e-2 and out["learned32"]["dq"] < 1e-4
