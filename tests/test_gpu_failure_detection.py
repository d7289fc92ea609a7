"""Failure detection without a GPU fault: a non-finite value planted in the
state on the host, a Newton iteration cap too small for the saturated nodes
of the moist layer, and a bounded tensor-core wait that runs out on a barrier
nothing arrives on (test hook).  Each is reported by cmles_diagnostics as a
status code (CMLES_ERR_NONFINITE, CMLES_ERR_SATADJ, CMLES_ERR_TIMEOUT) with
the context left usable: afterwards the next report is clean."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ERR_SATADJ, ERR_NONFINITE, ERR_TIMEOUT = 4, 5, 8


def _levels(arr, mesh):
    Nq = mesh["N"] + 1
    return np.array([arr[ez * mesh["nex"] * mesh["ney"], k * Nq * Nq] for ez in range(mesh["nez"])
                     for k in range(Nq)])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonfinite_state_is_reported_and_cleared(orc, precision):
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 3, 3, 8)
    ph = I.physics("c2")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    G = cmles.Solver(m, ph, precision=precision)
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    bad = Q.copy()
    bad[3, 4, 17] = np.nan
    G.set_state(torch.from_numpy(bad).cuda())
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == ERR_NONFINITE and d["nonfinite"]
    with pytest.raises(cmles.CmlesError):
        G.diagnostics()
    G.set_state(torch.from_numpy(Q).cuda())
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == 0 and not d["nonfinite"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_newton_cap_failures_are_counted(orc, precision):
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 5, 3, 16)
    ph = I.physics("c2")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    S.rhs(Q)
    assert (S.intermediates()["aux"][:, 3] > 0).mean() > 0.1          # saturated nodes present
    ph1 = dict(ph, satadj_max_iter=1)
    G = cmles.Solver(m, ph1, precision=precision)
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    G.tendency(torch.from_numpy(Q).cuda())
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == ERR_SATADJ and d["satadj_failures"] > 0
    # the counter is cleared by the report; the default cap converges
    G2 = cmles.Solver(m, ph, precision=precision)
    G2.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    G2.tendency(torch.from_numpy(Q).cuda())
    d2 = G2.diagnostics(raise_on_error=False)
    assert d2["status"] == 0 and d2["satadj_failures"] == 0
    d = G.diagnostics(raise_on_error=False)
    assert d["satadj_failures"] == 0


def test_newton_cap_failures_are_counted_in_the_flux_pass(orc):
    """On flat meshes the FP32 path runs the thermodynamics in the kernel that
    writes a state: the shadow kernel, and the flux pass for the state each
    stage advances to.  With the Newton cap at one iteration both count: a
    step (one shadow write, then five flux passes) reports more failures than
    a tendency call (one shadow write alone)."""
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 5, 3, 16)
    ph = dict(I.physics("c2"), satadj_max_iter=1)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    G = cmles.Solver(m, ph, precision="fp32")
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    G.tendency(torch.from_numpy(Q).cuda())
    n_shadow = G.diagnostics(raise_on_error=False)["satadj_failures"]
    assert n_shadow > 0
    G.set_state(torch.from_numpy(Q).cuda())
    G.step(1)
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == ERR_SATADJ and d["satadj_failures"] > n_shadow, (d["satadj_failures"], n_shadow)


def test_tensor_core_wait_timeout_is_reported_and_cleared(orc):
    """The learned-closure gradient pass bounds its waits on the tensor-core
    completion barrier.  A test hook adds a bounded wait on a barrier that
    nothing arrives on: the wait runs out, every CTA still finishes and frees
    its Tensor Memory, cmles_diagnostics reports CMLES_ERR_TIMEOUT with the
    count, and with the hook off the next report is clean.  The hook does not
    touch the network's own waits, so the tendency is unchanged."""
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 4, 3, 8)
    ph = I.physics("c2", closure="mlp")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    rng = np.random.default_rng(3)
    G = cmles.Solver(m, ph, precision="fp32")
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    flat = np.concatenate([rng.normal(size=5186) * 0.1, np.ones(13), [1.0, 1.0]]).astype(np.float32)
    G.set_closure_weights(flat)
    Qd = torch.from_numpy(Q).cuda()
    R0 = G.tendency(Qd).cpu().numpy()
    assert G.diagnostics(raise_on_error=False)["status"] == 0
    G.test_stall_tc(True)
    R1 = G.tendency(Qd).cpu().numpy()
    d = G.diagnostics(raise_on_error=False)
    # one CTA per element here (96 elements, fewer than the persistent grid),
    # each counted once
    assert d["status"] == ERR_TIMEOUT and d["tc_timeouts"] == G.E, (d["tc_timeouts"], G.E)
    assert np.array_equal(R1, R0)
    G.test_stall_tc(False)
    R2 = G.tendency(Qd).cpu().numpy()
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == 0 and d["tc_timeouts"] == 0
    assert np.array_equal(R2, R0)


def test_tensor_core_drain_after_a_wait_gives_up(orc):
    """A CTA whose MMA completion wait gives up while its MMA is still in
    flight (test hook mode 2: the first wait of each CTA makes no try) issues
    no further MMA, reads no Tensor Memory, and at its tear-down waits
    (bounded) for that MMA's completion before freeing the columns.  The launch reports
    CMLES_ERR_TIMEOUT with every CTA counted once; the context stays usable
    and the next tendency, with the hook off, is bit-identical to one taken
    before (its CTAs allocate the same Tensor Memory columns)."""
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 4, 3, 8)
    ph = I.physics("c2", closure="mlp")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    rng = np.random.default_rng(5)
    G = cmles.Solver(m, ph, precision="fp32")
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    flat = np.concatenate([rng.normal(size=5186) * 0.1, np.ones(13), [1.0, 1.0]]).astype(np.float32)
    G.set_closure_weights(flat)
    Qd = torch.from_numpy(Q).cuda()
    R0 = G.tendency(Qd).cpu().numpy()
    assert G.diagnostics(raise_on_error=False)["status"] == 0
    for _ in range(2):
        G.test_stall_tc(2)
        G.tendency(Qd)
        d = G.diagnostics(raise_on_error=False)
        assert d["status"] == ERR_TIMEOUT and d["tc_timeouts"] == G.E, (d["tc_timeouts"], G.E)
        G.test_stall_tc(0)
        R2 = G.tendency(Qd).cpu().numpy()
        d = G.diagnostics(raise_on_error=False)
        assert d["status"] == 0 and d["tc_timeouts"] == 0
        assert np.array_equal(R2, R0)
    with pytest.raises(cmles.CmlesError):
        G.test_stall_tc(3)


def test_tensor_core_wait_timeout_with_several_row_tiles(orc):
    """The same bounded wait in the learned pass above N = 4 (224-thread
    CTAs, two 128-row tiles and 128 Tensor Memory columns each): every CTA
    counted once, the tendency unchanged, the next report clean; mode 2,
    whose test instance is built for 128-thread CTAs, is refused."""
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 3, 2, 4, N=5)
    ph = I.physics("c2", closure="mlp")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    rng = np.random.default_rng(6)
    G = cmles.Solver(m, ph, precision="fp32")
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    flat = np.concatenate([rng.normal(size=5186) * 0.1, np.ones(13), [1.0, 1.0]]).astype(np.float32)
    G.set_closure_weights(flat)
    Qd = torch.from_numpy(Q).cuda()
    R0 = G.tendency(Qd).cpu().numpy()
    assert G.diagnostics(raise_on_error=False)["status"] == 0
    G.test_stall_tc(1)
    R1 = G.tendency(Qd).cpu().numpy()
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == ERR_TIMEOUT and d["tc_timeouts"] == G.E, (d["tc_timeouts"], G.E)
    assert np.array_equal(R1, R0)
    G.test_stall_tc(0)
    R2 = G.tendency(Qd).cpu().numpy()
    d = G.diagnostics(raise_on_error=False)
    assert d["status"] == 0 and d["tc_timeouts"] == 0
    assert np.array_equal(R2, R0)
    with pytest.raises(cmles.CmlesError):
        G.test_stall_tc(2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_condensate_below_freezing_is_counted_not_an_error(orc, precision):
    """The saturation adjustment keeps all condensate liquid (no ice phase).
    A node that condenses below 273.15 K is counted in cold_saturated, for
    information; the status stays CMLES_OK.  The stratified throughput box
    saturates only near its lid (the oracle's q_l > 0 nodes there are all
    colder than 202 K); the moist layer saturates only where it is warmer
    than 283 K, and counts nothing.  Both a tendency call and a step report
    (on the FP32 path the shadow kernel and the flux pass each count)."""
    from paper_2110_00853_b300 import cmles
    for name, dims, cold in (("c5", (2, 2, 80), True), ("c2", (3, 3, 16), False)):
        m = I.sub_mesh(name, *dims)
        ph = I.physics(name)
        S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case(name))
        S.rhs(Q)
        aux = S.intermediates()["aux"]
        sat = aux[:, 3] > 0
        assert sat.sum() > 1000
        T = aux[:, 2][sat]
        assert (T.max() < 273.15 - 50.0) if cold else (T.min() > 273.15 + 10.0)
        G = cmles.Solver(m, ph, precision=precision)
        G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
        G.tendency(torch.from_numpy(Q).cuda())
        d = G.diagnostics(raise_on_error=False)
        assert d["status"] == 0 and d["satadj_failures"] == 0
        assert (d["cold_saturated"] > 0) == cold, (name, d["cold_saturated"])
        G.set_state(torch.from_numpy(Q).cuda())
        G.step(1)
        d = G.diagnostics(raise_on_error=False)
        assert d["status"] == 0 and (d["cold_saturated"] > 0) == cold, (name, d["cold_saturated"])
        assert G.diagnostics(raise_on_error=False)["cold_saturated"] == 0    # cleared by the report
