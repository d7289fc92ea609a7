"""Host round trips through the C ABI: the asynchronous chunked download of
the state (cmles_fetch_state_host / cmles_wait_fetch) and the staged upload
of the same host buffer, which sends each chunk as soon as it has arrived.
Checked bit for bit against the synchronous host copies and against a run
that never leaves the device, with the orderings the download promises: a
step queued right after a download does not change what it delivers, and a
set or get of the same host buffer waits for it."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _levels(arr, mesh):
    Nq = mesh["N"] + 1
    return np.array([arr[ez * mesh["nex"] * mesh["ney"], k * Nq * Nq] for ez in range(mesh["nez"])
                     for k in range(Nq)])


def _solver(orc, precision, dims):
    from paper_2110_00853_b300 import cmles
    m, ph = I.sub_mesh("c2", *dims), I.physics("c2")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    G = cmles.Solver(m, ph, precision=precision)
    G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    return G, torch.from_numpy(Q)


def _pinned(like):
    return torch.empty(like.shape, dtype=torch.float64, pin_memory=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fetch_equals_get_state_host(orc, precision):
    # 5 x 3 x 16 elements: 180,000 doubles, so the 32 chunks are ragged
    G, Q = _solver(orc, precision, (5, 3, 16))
    G.set_state(Q.cuda())
    G.step(1)
    a = G.get_state_host()
    b = _pinned(a)
    G.fetch_state_host(b)
    G.wait_fetch()
    assert torch.equal(a, b)
    G.wait_fetch()                      # nothing pending: returns at once
    G.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pipelined_host_loop_equals_device_loop(orc, precision):
    """stage (chunk-chained with the previous download) -> commit -> step ->
    fetch, four times, ends where four steps on the device end."""
    G, Q = _solver(orc, precision, (4, 4, 16))
    G.set_state(Q.cuda())
    G.step(4)
    ref = G.get_state().cpu()
    G.close()
    G, Q = _solver(orc, precision, (4, 4, 16))
    bufs = [Q.clone().pin_memory(), _pinned(Q)]
    for k in range(4):
        G.stage_state_host(bufs[k % 2])
        G.commit_staged_state()
        G.step(1)
        G.fetch_state_host(bufs[(k + 1) % 2])
        d = G.diagnostics(raise_on_error=False)
        assert d["status"] == 0
    G.wait_fetch()
    assert torch.equal(bufs[0], ref)
    assert torch.equal(G.get_state().cpu(), ref)
    G.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_work_queued_after_a_download_is_ordered_after_it(orc, precision):
    """The whole moist layer (98 MB of state): a download followed at once
    by three steps delivers the state before the steps, and the steps run
    from that state; set_state_host and get_state_host of the buffer being
    downloaded into wait for the download."""
    G, Q = _solver(orc, precision, (32, 32, 16))
    G.set_state(Q.cuda())
    G.step(1)
    before = G.get_state().cpu()
    out = _pinned(Q)
    G.fetch_state_host(out)
    G.step(3)                           # queued while the download runs
    G.wait_fetch()
    assert torch.equal(out, before)
    after = G.get_state().cpu()
    G.set_state(before.cuda())
    G.step(3)
    assert torch.equal(G.get_state().cpu(), after)
    # set_state_host of the buffer being written waits for the download
    buf = _pinned(Q)
    buf.zero_()
    G.fetch_state_host(buf)
    G.set_state_host(buf)
    assert torch.equal(G.get_state().cpu(), after)
    # get_state_host into it as well (both write the same state)
    G.fetch_state_host(buf)
    G.get_state_host(out=buf)
    G.wait_fetch()
    assert torch.equal(buf, after)
    # closing the handle with a download in flight finishes the download
    last = _pinned(Q)
    G.fetch_state_host(last)
    G.close()
    assert torch.equal(last, after)
