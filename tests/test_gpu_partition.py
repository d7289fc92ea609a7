"""The domain decomposition on one GPU (cmles_group): a mesh split into
px x py (x, y) partitions, each with its own device buffers and a ring of
ghost elements that two halo exchanges per stage fill (state and
thermodynamic fields before the gradient pass, F2 before the flux pass).

Every element then runs the same kernels on the same values as in the whole
mesh's handle, so tendencies and steps must be bit-identical to it, on both
precisions, every closure, walls and periodic boundaries, uneven splits and a
partition that is its own neighbour across a periodic boundary; budgets are
summed over partitions (the allreduce of a multi-GPU run) and agree to
rounding.  One case is also compared with the FP64 oracle directly.
"""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _levels(arr, mesh):
    Nq = mesh["N"] + 1
    return np.array([arr[ez * mesh["nex"] * mesh["ney"], k * Nq * Nq] for ez in range(mesh["nez"])
                     for k in range(Nq)])


def _fuzz(Q, seed, amp_u=3.0, amp_rho=1e-3, amp_e=50.0):
    rng = np.random.default_rng(seed)
    Q = Q.copy()
    rho = Q[:, 0]
    u = rng.uniform(-amp_u, amp_u, size=(Q.shape[0], 3, Q.shape[2]))
    Q[:, 4] += 0.5 * rho * (u ** 2).sum(axis=1) + (Q[:, 1:4] * u).sum(axis=1)
    Q[:, 1:4] += rho[:, None] * u
    Q[:, 0] *= 1.0 + rng.uniform(-amp_rho, amp_rho, size=rho.shape)
    Q[:, 4] += rng.uniform(-amp_e, amp_e, size=rho.shape)
    return Q


def _weights(seed=7):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.normal(size=5186) * 0.1, [100.0] * 9 + [300.0] * 3 + [0.02], [5.0, 10.0]]
                          ).astype(np.float32)


def _pair(orc, mesh, phys, case, precision, px, py, fuzz_seed):
    from paper_2110_00853_b300 import cmles
    S, Q, rr, pr, _ = orc.from_inputs(mesh, phys, case)
    Q = _fuzz(Q, fuzz_seed)
    ref = (_levels(rr, mesh), _levels(pr, mesh), _levels(Q[:, 5] / Q[:, 0], mesh) if phys.get("moist") else None)
    W = cmles.Solver(mesh, phys, precision=precision)
    G = cmles.Group(mesh, phys, px, py, precision=precision)
    W.set_reference(*ref)
    G.set_reference(*ref)
    if phys.get("closure") == "mlp":
        W.set_closure_weights(_weights())
        G.set_closure_weights(_weights())
    return S, Q, W, G


CASES = [
    # name, mesh, precision, closure, split
    ("moist layer, periodic x y", I.sub_mesh("c2", 6, 5, 4), "fp64", "sl", (2, 1)),
    ("moist layer, uneven 3 x 2", I.sub_mesh("c2", 7, 5, 3), "fp64", "vreman", (3, 2)),
    ("moist layer, own neighbour in y", I.sub_mesh("c2", 6, 3, 3), "fp64", "sl", (3, 1)),
    ("moist layer, fp32", I.sub_mesh("c2", 6, 5, 4), "fp32", "sl", (2, 2)),
    ("moist layer, fp32 learned closure", I.sub_mesh("c2", 5, 6, 3), "fp32", "mlp", (2, 3)),
    ("moist layer, fp32 tiled partitions", I.sub_mesh("c2", 8, 8, 2), "fp32", "sl", (2, 2)),
    # walls in z with the drag law and no-slip ghosts, which every partition holds
    ("moist layer, fp64 no-slip and drag", I.sub_mesh("c2", 6, 4, 3), "fp64", "sl+walls", (3, 2)),
    ("moist layer, fp32 no-slip and drag", I.sub_mesh("c2", 8, 4, 3), "fp32", "sl+walls", (2, 2)),
    # orders above 4: CTAs of more than 128 threads, FP32 arrays padded to np32(N) nodes
    ("moist layer, fp32 order 5", I.sub_mesh("c2", 4, 4, 3, N=5), "fp32", "sl", (2, 2)),
    ("moist layer, fp32 learned closure order 6", I.sub_mesh("c2", 4, 3, 2, N=6), "fp32", "mlp", (2, 1)),
    ("moist layer, fp64 order 7", I.sub_mesh("c2", 4, 3, 2, N=7), "fp64", "vreman", (2, 3)),
]


@pytest.mark.parametrize("label,mesh,precision,closure,split", CASES, ids=[c[0] for c in CASES])
def test_group_tendency_and_steps_are_bit_identical(orc, label, mesh, precision, closure, split):
    if closure == "sl+walls":
        phys = dict(I.physics("c2", closure="sl"), drag_cd=0.015, noslip=0b110000)
    else:
        phys = I.physics("c2", closure=closure)
    S, Q, W, G = _pair(orc, mesh, phys, I.case("c2"), precision, *split, fuzz_seed=3)
    Qd = torch.from_numpy(Q).cuda()
    Rw = W.tendency(Qd).cpu().numpy()
    Rg = G.tendency(Qd).cpu().numpy()
    assert np.array_equal(Rg, Rw), (label, np.abs(Rg - Rw).max())
    assert G.halo_bytes() > 0
    W.set_state(Qd)
    G.set_state(Qd)
    for _ in range(2):
        W.step(1)
        G.step(1)
        Qw = W.get_state().cpu().numpy()
        Qg = G.get_state().cpu().numpy()
        assert np.array_equal(Qg, Qw), (label, np.abs(Qg - Qw).max())
    dw, dg = W.diagnostics(raise_on_error=False), G.diagnostics(raise_on_error=False)
    assert dw["status"] == 0 and dg["status"] == 0
    assert np.allclose(dg["budget"], dw["budget"], rtol=1e-14, atol=0.0), (dg["budget"], dw["budget"])
    assert dg["steps"] == 2
    W.close()
    G.close()


def test_group_walls_and_lateral_sponge(orc):
    """Walls at both x ends (no exchange there) and the lateral sponge, whose
    columns each partition takes from the whole mesh's table."""
    mesh = dict(I.sub_mesh("c2", 9, 4, 3), periodic=(0, 1, 0))
    phys = dict(I.physics("c2"), lateral_sponge_frac=0.2, sponge_alpha=0.5, u_relax=(2.0, 0.0, 0.0))
    for precision in ("fp64", "fp32"):
        S, Q, W, G = _pair(orc, mesh, phys, I.case("c2"), precision, 3, 2, fuzz_seed=5)
        Qd = torch.from_numpy(Q).cuda()
        assert np.array_equal(G.tendency(Qd).cpu().numpy(), W.tendency(Qd).cpu().numpy()), precision
        W.set_state(Qd)
        G.set_state(Qd)
        W.step(2)
        G.step(2)
        assert np.array_equal(G.get_state().cpu().numpy(), W.get_state().cpu().numpy()), precision
        if precision == "fp64":
            R_orc, fails = S.rhs(Q)
            assert fails == 0
            Rg = G.tendency(Qd).cpu().numpy()
            for v in range(6):
                err = np.linalg.norm(Rg[:, v] - R_orc[:, v]) / np.linalg.norm(R_orc[:, v])
                assert err <= 1e-12, (v, err)
        W.close()
        G.close()


def test_group_rejects_what_it_does_not_run():
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 4, 4, 2)
    with pytest.raises(cmles.CmlesError):
        cmles.Group(m, I.physics("c2"), 5, 1)
    with pytest.raises(cmles.CmlesError):
        cmles.Group(m, dict(I.physics("c2"), integrator="ark2_hevi"), 2, 1)
    with pytest.raises(cmles.CmlesError):
        cmles.Group(m, dict(I.physics("c2"), filter_order=16), 2, 1)
