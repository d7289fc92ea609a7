"""GPU parity on the warped terrain-following mesh (the flow-over-hill
configuration: Gaussian ridge, constant Brunt-Vaisala frequency, 10 m/s
inflow, lateral and top sponge) for the FP32 path with FP64 accumulation,
against the FP64 CPU oracle, which evaluates the same mesh with its own
curl-form metric terms."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _hill_box(nex=8, ney=2, nez=8, N=4):
    # a window of the hill configuration's element size around the ridge
    h = 40000.0 / 128
    return dict(N=N, nex=nex, ney=ney, nez=nez, Lx=nex * h, Ly=ney * h, Lz=nez * h, x0=20000.0 - nex * h / 2,
                y0=0.0, z0=0.0, periodic=(1, 1, 0), warp=True, hill_h=400.0, hill_a=1000.0, hill_xc=20000.0)


def _phys(m):
    ph = I.physics("c3")
    ph.update(sponge_zs=0.75 * m["Lz"])
    return ph


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _setup(orc, fuzz=True, flux="rusanov", N=4, box=(8, 2, 8), dt=None, closure="sl"):
    from paper_2110_00853_b300 import cmles
    m = _hill_box(*box, N=N)
    ph = _phys(m)
    ph["flux"] = flux
    ph["closure"] = closure
    if dt is not None:
        ph["dt"] = dt
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c3"))
    if fuzz:
        rng = np.random.default_rng(31)
        u = rng.uniform(-2.0, 2.0, size=(Q.shape[0], 3, Q.shape[2]))
        Q = Q.copy()
        Q[:, 4] += 0.5 * Q[:, 0] * (u ** 2).sum(1) + (Q[:, 1:4] * u).sum(1)
        Q[:, 1:4] += Q[:, 0][:, None] * u
        Q[:, 4] += rng.uniform(-20.0, 20.0, size=Q[:, 4].shape)
    G = cmles.Solver(m, ph, precision="fp32")
    G.set_reference(rr.ravel(), pr.ravel(), None)
    return m, S, Q, G


@pytest.mark.parametrize("flux", ["rusanov", "hllc", "roe"])
def test_warped_tendency_parity(orc, flux):
    m, S, Q, G = _setup(orc, flux=flux)
    J = S.geometry()["J"]
    assert J.std() / J.mean() > 1e-2          # genuinely curved elements
    R_orc, _ = S.rhs(Q)
    R_gpu = G.tendency(torch.from_numpy(Q).cuda()).cpu().numpy()
    errs = [_rel(R_gpu[:, v], R_orc[:, v]) for v in range(5)]
    print("warped fp32", flux, "rel L2", errs)
    for v in range(5):
        assert errs[v] <= 1e-5, (v, errs)
        # node by node as well (a wrong value on a few nodes can hide in the norm)
        assert np.abs(R_gpu[:, v] - R_orc[:, v]).max() <= 1e-4 * np.abs(R_orc[:, v]).max(), v


def test_warped_initial_state_matches_oracle(orc):
    from paper_2110_00853_b300 import cmles
    m = _hill_box()
    ph = _phys(m)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c3"))
    G = cmles.Solver(m, ph, precision="fp32")
    G.init_case(I.case("c3"))
    Qg = G.get_state().cpu().numpy()
    for v in range(5):
        assert np.abs(Qg[:, v] - Q[:, v]).max() <= 1e-12 * np.abs(Q[:, v]).max(), v


def test_warped_steps_track_oracle_and_conserve(orc):
    m, S, Q, G = _setup(orc)
    n, dt = 4, 0.02
    Q_orc, _ = S.lsrk54(Q, n, dt)
    G.set_state(torch.from_numpy(Q).cuda())
    b0 = G.diagnostics()["budget"]
    G.step(n)
    Qg = G.get_state().cpu().numpy()
    b1 = G.diagnostics()["budget"]
    for v in range(5):
        e = _rel(Qg[:, v] - Q[:, v], Q_orc[:, v] - Q[:, v])
        print("warped 4-step increment rel L2", v, e)
        assert e <= 1e-5, v
    bo, _ = S.budgets(Q)
    assert np.allclose(b0, bo, rtol=1e-13)
    for v in (0, 4):     # walls and periodic sides: mass and energy conserved
        assert abs(b1[v] - b0[v]) <= 1e-10 * abs(b0[v]), v


@pytest.mark.parametrize("N", [4, 6])
def test_warped_free_stream(orc, N):
    from paper_2110_00853_b300 import cmles
    m = _hill_box(N=N)
    ph = _phys(m)
    ph.update(g=0.0, sponge_alpha=0.0)
    G = cmles.Solver(m, ph, precision="fp32")
    E, Np = G.E, G.Np
    rho, T, u = 1.2, 300.0, np.array([10.0, 2.0, 0.0])
    p = rho * 287.0 * T
    Q = np.zeros((E, 6, Np))
    Q[:, 0] = rho
    Q[:, 1:4] = (rho * u)[None, :, None]
    Q[:, 4] = rho * (717.5 * (T - 273.16) + 0.5 * u @ u)
    G.set_reference(np.full(E * Np, rho), np.full(E * Np, p), None)
    R = G.tendency(torch.from_numpy(Q).cuda()).cpu().numpy()
    ez = np.arange(E) // (m["nex"] * m["ney"])
    inner = (ez > 0) & (ez < m["nez"] - 1)
    # interior elements see no walls: the uniform flow stays uniform up to FP32 rounding
    assert np.abs(R[inner][:, 1:4]).max() < 1e-5 * rho * 100.0 / 100.0


@pytest.mark.parametrize("N,flux,closure", [(2, "rusanov", "sl"), (3, "hllc", "sl"), (5, "rusanov", "sl"),
                                            (6, "roe", "sl"), (7, "rusanov", "sl"), (4, "rusanov", "vreman"),
                                            (5, "hllc", "vreman")])
def test_warped_other_orders_tendency_and_steps(orc, N, flux, closure):
    """The curvilinear FP32 kernels at orders other than 4 (above 4: CTAs of
    np32(N) threads, arrays and metric tables padded to as many nodes), and
    with the Vreman closure (each curved element's directional lengths: its
    nodes' extent along x, y, z over N), on a window around the ridge: the
    tendency against the oracle's, in norm and node by node, then four steps,
    with mass and energy conserved."""
    dt = 0.02 * min(1.0, (4.0 / N) ** 2)      # the step shrinks with the smallest node spacing
    m, S, Q, G = _setup(orc, flux=flux, N=N, box=(8, 2, 8) if N <= 4 else (6, 2, 6), dt=dt, closure=closure)
    R_orc, _ = S.rhs(Q)
    assert S.intermediates()["nut"].max() > 0.0      # the closure is active
    R_gpu = G.tendency(torch.from_numpy(Q).cuda()).cpu().numpy()
    errs = [_rel(R_gpu[:, v], R_orc[:, v]) for v in range(5)]
    print("warped fp32 N", N, flux, closure, "rel L2", errs)
    for v in range(5):
        assert errs[v] <= 1e-5, (v, errs)
        assert np.abs(R_gpu[:, v] - R_orc[:, v]).max() <= 1e-4 * np.abs(R_orc[:, v]).max(), v
    n = 4
    Q_orc, _ = S.lsrk54(Q, n, dt)
    G.set_state(torch.from_numpy(Q).cuda())
    b0 = G.diagnostics()["budget"]
    G.step(n)
    Qg = G.get_state().cpu().numpy()
    b1 = G.diagnostics()["budget"]
    G.close()
    for v in range(5):
        e = _rel(Qg[:, v] - Q[:, v], Q_orc[:, v] - Q[:, v])
        print("warped N", N, "4-step increment rel L2", v, e)
        assert e <= 1e-5, v
    for v in (0, 4):
        assert abs(b1[v] - b0[v]) <= 1e-10 * abs(b0[v]), v


@pytest.mark.parametrize("N", [4, 6])
def test_warped_tendency_with_learned_closure(orc, N):
    """The curvilinear gradient pass with the learned closure on the tcgen05
    tensor cores (BF16 network, per-node Delta of the curved elements)
    against the oracle's BF16-defined network: bound 1e-4 relative L2, as
    on the flat mesh (a hidden activation can round to the neighbouring BF16
    value).  At N = 6 each element's 343 rows are three tiles of 128 rows
    (three MMA chains per layer, TMEM column blocks 0, 64, 128)."""
    from paper_2110_00853_b300 import cmles
    m = _hill_box(N=N) if N <= 4 else _hill_box(6, 2, 6, N=N)
    ph = _phys(m)
    ph["closure"] = "mlp"
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c3"))
    rng = np.random.default_rng(32)
    u = rng.uniform(-2.0, 2.0, size=(Q.shape[0], 3, Q.shape[2]))
    Q = Q.copy()
    Q[:, 4] += 0.5 * Q[:, 0] * (u ** 2).sum(1) + (Q[:, 1:4] * u).sum(1)
    Q[:, 1:4] += Q[:, 0][:, None] * u
    bf = np.vectorize(orc.bf16)
    W = {"W1": bf(rng.normal(size=(64, 13)) * 0.3), "b1": rng.normal(size=64).astype(np.float32) * 0.1,
         "W2": bf(rng.normal(size=(64, 64)) * 0.15), "b2": rng.normal(size=64).astype(np.float32) * 0.1,
         "W3": bf(rng.normal(size=(2, 64)) * 0.1), "b3": np.array([0.7, 0.5], np.float32)}
    W = {k: np.asarray(v, np.float64) for k, v in W.items()}
    in_scale, out_scale = np.array([1.0] * 9 + [30.0] * 3 + [0.02]), np.array([20.0, 40.0])
    S.set_mlp(W, in_scale, out_scale)
    R_orc, _ = S.rhs(Q)
    assert S.intermediates()["nut"].max() > 1.0
    flat = np.concatenate([W[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")] +
                          [in_scale, out_scale]).astype(np.float32)
    G = cmles.Solver(m, ph, precision="fp32")
    G.set_reference(rr.ravel(), pr.ravel(), None)
    G.set_closure_weights(flat)
    R_gpu = G.tendency(torch.from_numpy(Q).cuda()).cpu().numpy()
    errs = [_rel(R_gpu[:, v], R_orc[:, v]) for v in range(5)]
    print("warped fp32 learned closure N", N, "rel L2", errs)
    assert G.diagnostics(raise_on_error=False)["status"] == 0
    for v in range(5):
        assert errs[v] <= 1e-4, (v, errs)
        assert np.abs(R_gpu[:, v] - R_orc[:, v]).max() <= 1e-3 * np.abs(R_orc[:, v]).max(), v


def test_warped_tendency_between_steps_leaves_the_state_alone(orc):
    """As on flat meshes: a tendency call between two steps (of another
    state) leaves the stepped state, its shadow and its thermodynamic fields
    alone; the result is bit-identical to two steps without it."""
    m, S, Q, G = _setup(orc)
    Qd = torch.from_numpy(Q).cuda()
    G.set_state(Qd)
    G.step(2)
    ref = G.get_state().cpu().numpy()
    G.set_state(Qd)
    G.step(1)
    G.tendency(torch.from_numpy(Q * (1.0 + 1e-4)).cuda())
    G.step(1)
    assert np.array_equal(G.get_state().cpu().numpy(), ref)
