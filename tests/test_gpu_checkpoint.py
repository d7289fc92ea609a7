"""Checkpoint and resume through the C ABI: a run interrupted after two steps,
saved to host memory, and continued on a fresh handle from that copy ends
bit-identical to the uninterrupted run.  Holds because a step starts from
the FP64 state alone: the first stage has A = 0 (no LSRK register is read),
and the FP32 path rebuilds its shadow and starts a new step increment from
the FP64 state."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _levels(arr, mesh):
    Nq = mesh["N"] + 1
    return np.array([arr[ez * mesh["nex"] * mesh["ney"], k * Nq * Nq] for ez in range(mesh["nez"])
                     for k in range(Nq)])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resume_from_host_checkpoint_is_bit_identical(orc, precision):
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c2", 4, 4, 16)
    ph = I.physics("c2")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    ref = (_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))

    def solver():
        G = cmles.Solver(m, ph, precision=precision)
        G.set_reference(*ref)
        return G

    A = solver()
    A.set_state(torch.from_numpy(Q).cuda())
    A.step(4)
    full = A.get_state().cpu()

    B = solver()
    B.set_state(torch.from_numpy(Q).cuda())
    B.step(2)
    saved = B.get_state_host().clone()
    B.close()

    C = solver()
    C.set_state_host(saved)
    C.step(2)
    resumed = C.get_state().cpu()
    assert torch.equal(full, resumed)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_staged_host_upload_equals_set_state(orc, precision):
    """cmles_stage_state_host + cmles_commit_staged_state take a host state
    exactly as cmles_set_state_host does (the step that follows is
    bit-identical), while the copy overlaps queued work; committing with
    nothing staged is an error."""
    from paper_2110_00853_b300 import cmles
    m, ph = I.sub_mesh("c2", 3, 3, 8), I.physics("c2")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    host = torch.from_numpy(Q).pin_memory()
    out = []
    for staged in (False, True):
        G = cmles.Solver(m, ph, precision=precision)
        G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
        G.set_state_host(host)
        if staged:
            with pytest.raises(cmles.CmlesError):
                G.commit_staged_state()
            G.step(1)
            G.stage_state_host(host)        # the copy overlaps the next queued step
            G.step(1)
            G.commit_staged_state()         # back to the host state
        G.step(2)
        out.append(G.get_state().cpu().numpy())
        G.close()
    assert np.array_equal(out[0], out[1])
