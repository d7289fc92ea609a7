"""Parity at full size: the throughput box (160 x 160 x 80 elements, N = 4,
256M nodes) built by the library's own initial-state kernel, evaluated by the
same kernels bench.py times, checked on sampled elements against the FP64
CPU oracle.

The right-hand side of an element depends on its face neighbours and on
theirs (the gradient pass reads neighbour faces, the flux pass reads the
neighbours' gradients), so the oracle evaluates a window of +-2 elements
around each sampled element and only the centre is compared; for one whole
LSRK(5,4) step the dependence reaches 2 elements per stage, so the window is
+-10 elements.  Walls are real boundaries of the box; the window's other
faces never influence the compared element.

As in the small parity tests the state carries seeded fuzz (velocity
+-3 m/s, density +-0.1 %, energy +-50 J m^-3, drawn on the GPU with a seeded
torch generator) so that every tendency is O(1); the unperturbed box has
p - p_r = 0 above the noise layer, where relative errors only measure
rounding of a near-zero tendency.  Tolerances as in the small tests: FP64
1e-12, FP32 with FP64 accumulation 1e-5 relative L2 per variable over the
sampled elements.
"""
import gc

import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAME = "c5"


def _window(full, ex, ey, ez, halo):
    """window mesh and the global element indices in window order"""
    n = (full["nex"], full["ney"], full["nez"])
    z0 = max(ez - halo, 0)
    z1 = min(ez + halo, n[2] - 1)
    hx, hy, hz = full["Lx"] / n[0], full["Ly"] / n[1], full["Lz"] / n[2]
    w = 2 * halo + 1
    m = dict(N=full["N"], nex=w, ney=w, nez=z1 - z0 + 1, Lx=w * hx, Ly=w * hy, Lz=(z1 - z0 + 1) * hz,
             x0=(ex - halo) * hx, y0=(ey - halo) * hy, z0=z0 * hz, periodic=(0, 0, 0), warp=False,
             hill_h=0.0, hill_a=1.0, hill_xc=0.0)
    idx = []
    for kz in range(z0, z1 + 1):
        for ky in range(ey - halo, ey + halo + 1):
            for kx in range(ex - halo, ex + halo + 1):
                idx.append((kx % n[0]) + n[0] * ((ky % n[1]) + n[1] * kz))
    centre = halo + w * (halo + w * (ez - z0))
    return m, np.array(idx), centre


def _oracle_window(orc, full, phys, case, Qw, m):
    c = dict(case)
    c["modes"] = None
    S, _, rr, pr, _ = orc.from_inputs(m, phys, c)
    S.set_reference(rr, pr)
    return S


def _samples(full):
    n = (full["nex"], full["ney"], full["nez"])
    rng = np.random.default_rng(123)
    pts = [(n[0] // 2, n[1] // 2, n[2] // 2), (0, 0, 0), (n[0] - 1, 3, n[2] - 1), (17, n[1] - 1, 1)]
    pts += [tuple(int(rng.integers(0, n[d])) for d in range(3)) for _ in range(2)]
    return pts


def _oracle_levels(orc, full, phys, case):
    """hydrostatic reference per node level of the full box from the
    oracle's own profile code (a one-column mesh of the same levels), so that
    both sides use identical reference values"""
    col = dict(full, nex=1, ney=1, Lx=full["Lx"] / full["nex"], Ly=full["Ly"] / full["ney"])
    c = dict(case)
    c["modes"] = None
    S, Q, rr, pr, _ = orc.from_inputs(col, phys, c)
    Nq = full["N"] + 1
    lev = lambda a: np.array([a[ez, k * Nq * Nq] for ez in range(full["nez"]) for k in range(Nq)])
    return lev(rr), lev(pr), lev(Q[:, 5] / Q[:, 0])


def _fuzz_gpu(Q, seed=77):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    rho = Q[:, 0]
    u = (torch.rand(Q[:, 1:4].shape, generator=g, device="cuda", dtype=torch.float64) * 2 - 1) * 3.0
    Q[:, 4] += 0.5 * rho * (u * u).sum(1) + (Q[:, 1:4] * u).sum(1)
    Q[:, 1:4] += rho[:, None] * u
    Q[:, 0] *= 1.0 + (torch.rand(rho.shape, generator=g, device="cuda", dtype=torch.float64) * 2 - 1) * 1e-3
    Q[:, 4] += (torch.rand(rho.shape, generator=g, device="cuda", dtype=torch.float64) * 2 - 1) * 50.0
    return Q


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _node_bound(got, want, tol, label):
    """Node by node: max |GPU - oracle| <= 10 tol max |oracle| (a wrong value
    on a few nodes can hide in a norm over many)."""
    err = np.abs(got - want).max()
    assert err <= 10 * tol * np.abs(want).max(), (label, err, np.abs(want).max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fullsize_tendency_sampled(orc, precision):
    from paper_2110_00853_b300 import cmles
    full, phys, case = I.mesh(NAME), I.physics(NAME), I.case(NAME)
    G = cmles.Solver(full, phys, precision=precision)
    G.init_case(case)
    G.set_reference(*_oracle_levels(orc, full, phys, case))
    Q = _fuzz_gpu(G.get_state())
    R = G.tendency(Q)
    torch.cuda.synchronize()
    got, want = [], []
    for (ex, ey, ez) in _samples(full):
        m, idx, centre = _window(full, ex, ey, ez, 2)
        Qw = Q[torch.from_numpy(idx).cuda()].cpu().numpy()
        S = _oracle_window(orc, full, phys, case, Qw, m)
        Rw, fails = S.rhs(Qw)
        assert fails == 0
        got.append(R[int(idx[centre])].cpu().numpy())
        want.append(Rw[centre])
    got, want = np.array(got), np.array(want)
    del Q, R
    G.close()
    gc.collect()
    torch.cuda.empty_cache()
    errs = [_rel(got[:, v], want[:, v]) for v in range(6)]
    print(precision, "full-size sampled tendency rel L2", errs)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for v in range(6):
        assert errs[v] <= tol, (v, errs)
        _node_bound(got[:, v], want[:, v], tol, v)


def test_fullsize_lsrk_step_sampled(orc):
    """one whole LSRK(5,4) step of the FP32 path at full size (the bench's
    timed configuration), compared on three +-10-element windows"""
    from paper_2110_00853_b300 import cmles
    full, phys, case = I.mesh(NAME), I.physics(NAME), I.case(NAME)
    G = cmles.Solver(full, phys, precision="fp32")
    G.init_case(case)
    G.set_reference(*_oracle_levels(orc, full, phys, case))
    Q0 = _fuzz_gpu(G.get_state())
    G.set_state(Q0)
    G.step(1)
    Q1 = G.get_state()
    pts = [(40, 100, 40), (5, 150, 0), (159, 0, 79)]
    errs = []
    for (ex, ey, ez) in pts:
        m, idx, centre = _window(full, ex, ey, ez, 10)
        sel = torch.from_numpy(idx).cuda()
        Qw0 = Q0[sel].cpu().numpy()
        S = _oracle_window(orc, full, phys, case, Qw0, m)
        Qw1, fails = S.lsrk54(Qw0, 1, phys["dt"])
        assert fails == 0
        d_gpu = Q1[int(idx[centre])].cpu().numpy() - Qw0[centre]
        d_orc = Qw1[centre] - Qw0[centre]
        errs.append([_rel(d_gpu[v], d_orc[v]) for v in range(6)])
    G.close()
    print("full-size one-step increment rel L2 per window", errs)
    for e in errs:
        for v in range(6):
            assert e[v] <= 1e-5, (v, e)


def test_fullsize_tendency_learned_closure(orc):
    """The headline configuration: the FP32 path with the learned closure on
    the full box, with the seeded network the benchmark uses, against the
    oracle's BF16-defined network on sampled +-2-element windows.  Bound as
    for the small learned-closure test: 1e-4 (BF16 activation flips reach
    nu_t directly)."""
    from paper_2110_00853_b300 import closure, cmles
    full, case = I.mesh(NAME), I.case(NAME)
    phys = I.physics(NAME, closure="mlp")
    p = closure.init_params(seed=0, in_scale=[100.0] * 9 + [300.0] * 3 + [0.02], out_scale=(5.0, 10.0),
                            b3=(0.5, 0.5)).astype(np.float64)
    shapes = (("W1", 64 * 13, True), ("b1", 64, False), ("W2", 64 * 64, True), ("b2", 64, False),
              ("W3", 2 * 64, True), ("b3", 2, False))
    W, o = {}, 0
    for k, n, is_w in shapes:
        v = p[o:o + n]
        W[k] = np.array([orc.bf16(x) for x in v]) if is_w else v.copy()
        o += n
    in_scale, out_scale = p[o:o + 13], p[o + 13:o + 15]
    flat = np.concatenate([W[k] for k, _, _ in shapes] + [in_scale, out_scale]).astype(np.float32)
    levels = _oracle_levels(orc, full, phys, case)
    G = cmles.Solver(full, phys, precision="fp32")
    G.init_case(case)
    G.set_reference(*levels)
    G.set_closure_weights(flat)
    Q = _fuzz_gpu(G.get_state())
    R = G.tendency(Q)
    torch.cuda.synchronize()
    pts = _samples(full)[:4]
    sel = []
    for (ex, ey, ez) in pts:
        m, idx, centre = _window(full, ex, ey, ez, 2)
        sel.append((m, idx, centre, Q[torch.from_numpy(idx).cuda()].cpu().numpy()))
    got = np.array([R[int(idx[c])].cpu().numpy() for (_, idx, c, _) in sel])
    del R
    G.close()
    # the same state without a closure isolates the closure's share of the tendency
    phys0 = dict(phys, closure="none")
    G0 = cmles.Solver(full, phys0, precision="fp32")
    G0.set_reference(*levels)
    R0 = G0.tendency(Q)
    got0 = np.array([R0[int(idx[c])].cpu().numpy() for (_, idx, c, _) in sel])
    del Q, R0
    G0.close()
    gc.collect()
    torch.cuda.empty_cache()
    want, want0 = [], []
    for (m, idx, centre, Qw) in sel:
        S = _oracle_window(orc, full, phys, case, Qw, m)
        S.set_mlp(W, in_scale, out_scale)
        Rw, fails = S.rhs(Qw)
        assert fails == 0
        want.append(Rw[centre])
        S0 = _oracle_window(orc, full, phys0, case, Qw, m)
        want0.append(S0.rhs(Qw)[0][centre])
    want, want0 = np.array(want), np.array(want0)
    errs = [_rel(got[:, v], want[:, v]) for v in range(6)]
    share = [np.linalg.norm(want[:, v] - want0[:, v]) / max(np.linalg.norm(want[:, v]), 1e-300) for v in range(6)]
    errs_c = [_rel(got[:, v] - got0[:, v], want[:, v] - want0[:, v]) for v in range(6)]
    print("full-size learned-closure tendency rel L2", errs)
    print("closure share of the tendency", share)
    print("closure contribution rel L2", errs_c)
    for v in range(6):
        assert errs[v] <= 1e-4, (v, errs)
        _node_bound(got[:, v], want[:, v], 1e-4, v)
    # the closure's own contribution (measured 3e-5 momentum, 4e-4 energy,
    # 2e-4 water): FP32 gradients and BF16 activation flips; the mass
    # equation's share (the water diffusion, 1e-5 of its tendency) is below
    # the FP32 rounding of the rest and is not compared
    for v in range(1, 6):
        assert errs_c[v] <= 1e-3, (v, errs_c)
