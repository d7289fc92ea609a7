"""The halo exchange of the domain decomposition on CPU, two gloo ranks: the
library's halo plan (cmles_halo_plan) drives a pack / point-to-point send and
receive / unpack between two partitions held as host arrays, and every ghost
node the DG kernels read across a partition boundary must then hold the
whole mesh's value; walls get no exchange, and a partition that spans a
periodic direction is its own neighbour there.  Also the plan's counts,
neighbours and index ranges on one process."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_halo_exchange(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "halo_worker.py"), str(tmp_path)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    recs = [json.load(open(tmp_path / f"halo{r}.json")) for r in range(2)]
    for rank, cases in enumerate(recs):
        for c in cases:
            assert c["rank"] == rank
            assert c["errors"] == 0 and c["checked"] > 0, c
            assert c["interior_intact"], c
            px, py, per = c["px"], c["py"], c["periodic"]
            nb = c["neighbours"]
            # x sides: the other rank, or a wall at the mesh's x ends when x is not periodic
            if px == 2:
                other = 1 - rank
                assert nb[0 if rank == 1 else 1] == other
                assert nb[1 if rank == 1 else 0] == (other if per[0] else -1)
                assert nb[2] == (rank if per[1] else -1) and nb[3] == (rank if per[1] else -1)
            else:
                other = 1 - rank
                assert nb[2 if rank == 1 else 3] == other
                assert nb[3 if rank == 1 else 2] == (other if per[1] else -1)
                assert nb[0] == (rank if per[0] else -1) and nb[1] == (rank if per[0] else -1)
            assert sorted(c["walls"]) == [s for s in range(4) if nb[s] < 0]


@pytest.mark.parametrize("N", [4, 7])
def test_halo_plan_counts_and_ranges(N):
    from paper_2110_00853_b300 import cmles
    mesh = dict(N=N, nex=7, ney=5, nez=3, Lx=7.0, Ly=5.0, Lz=3.0, periodic=(1, 0, 0))
    Np, Nf = (N + 1) ** 3, (N + 1) ** 2
    total_send = 0
    for rank in range(3 * 2):
        nb, cnt, send, recv = cmles.halo_plan(mesh, 3, 2, rank)
        ix, iy = rank % 3, rank // 3
        nx = [3, 2, 2][ix]
        ny = [3, 2][iy]
        Es = (nx + 2) * (ny + 2) * 3
        assert nb[0] == (ix - 1) % 3 + 3 * iy and nb[1] == (ix + 1) % 3 + 3 * iy
        assert nb[2] == (-1 if iy == 0 else rank - 3) and nb[3] == (-1 if iy == 1 else rank + 3)
        for s in range(4):
            along = ny if s < 2 else nx
            assert cnt[s] == (0 if nb[s] < 0 else 3 * along * Nf)
            if cnt[s]:
                assert send[s].min() >= 0 and send[s].max() < Es * Np
                assert recv[s].min() >= 0 and recv[s].max() < Es * Np
                assert len(np.unique(send[s])) == cnt[s] and len(np.unique(recv[s])) == cnt[s]
                # what side s sends, the neighbour receives on its side s ^ 1, entry for entry
                nb_nb, nb_cnt, _, _ = cmles.halo_plan(mesh, 3, 2, nb[s])
                assert nb_nb[s ^ 1] == rank and nb_cnt[s ^ 1] == cnt[s]
        total_send += sum(cnt)
    assert total_send > 0
    for bad in ((0, 1, 0), (8, 1, 0), (3, 2, 6), (3, 6, 0)):
        try:
            cmles.halo_plan(mesh, *bad)
        except cmles.CmlesError:
            continue
        raise AssertionError(bad)
