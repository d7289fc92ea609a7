"""Worker of the two-rank CPU test of the halo exchange (gloo): each rank
owns one partition of a small mesh as host arrays in the partition's storage
layout (interior plus one ghost element on each side in x and y), packs its
sides with the library's halo plan (cmles_halo_plan), exchanges them with its
neighbours by point-to-point send/receive, unpacks them into its ghost
elements and checks them against the whole mesh's values.  Launched by
tests/test_halo_cpu.py under torch.distributed.run."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

from paper_2110_00853_b300 import cmles  # noqa: E402


def split(n, parts, idx):
    base, extra = divmod(n, parts)
    return idx * base + min(idx, extra), base + (1 if idx < extra else 0)


def run_case(mesh, px, py, rank, world):
    N = mesh["N"]
    Nq, Np = N + 1, (N + 1) ** 3
    nex, ney, nez = mesh["nex"], mesh["ney"], mesh["nez"]
    # whole-mesh values: distinct per (element, variable, node)
    G = (np.arange(nex * ney * nez * 6 * Np, dtype=np.float64) + 0.25).reshape(nex * ney * nez, 6, Np)
    ix, iy = rank % px, rank // px
    x0, nx = split(nex, px, ix)
    y0, ny = split(ney, py, iy)
    Es = (nx + 2) * (ny + 2) * nez
    L = np.full((Es, 6, Np), np.nan)

    def sidx(ex, ey, ez):
        return (ex + 1) + (nx + 2) * ((ey + 1) + (ny + 2) * ez)

    for ez in range(nez):
        for ey in range(ny):
            for ex in range(nx):
                L[sidx(ex, ey, ez)] = G[(x0 + ex) + nex * ((y0 + ey) + ney * ez)]
    nb, cnt, send, recv = cmles.halo_plan(mesh, px, py, rank)
    Lf = L.reshape(Es, 6, Np)
    bufs = {}
    for s in range(4):
        if nb[s] < 0:
            continue
        e, n = np.divmod(send[s], Np)
        bufs[s] = torch.from_numpy(np.ascontiguousarray(Lf[e, :, n]))  # [count][6]
    # point-to-point exchange: side s goes to nb[s], which receives it on s ^ 1
    reqs, incoming = [], {}
    for s in range(4):
        if nb[s] < 0:
            continue
        incoming[s] = torch.empty((cnt[s], 6), dtype=torch.float64)
        if nb[s] == rank:
            continue
        reqs.append(dist.isend(bufs[s], dst=nb[s], tag=s))
        reqs.append(dist.irecv(incoming[s], src=nb[s], tag=s ^ 1))
    for r in reqs:
        r.wait()
    for s in range(4):
        if nb[s] == rank:  # across a periodic boundary the partition is its own neighbour
            incoming[s].copy_(bufs[s ^ 1])
    for s in incoming:
        e, n = np.divmod(recv[s], Np)
        Lf[e, :, n] = incoming[s].numpy()
    # every ghost node a kernel reads must now hold the neighbour element's value
    errors, checked = 0, 0
    for s in range(4):
        d, hi = s >> 1, s & 1
        if nb[s] < 0:
            continue
        a_nb = 0 if hi else N  # the node a kernel reads in the element across side s
        along = ny if d == 0 else nx
        for ez in range(nez):
            for p in range(along):
                gx = (nx if hi else -1) if d == 0 else p
                gy = p if d == 0 else (ny if hi else -1)
                gex, gey = (x0 + gx) % nex, (y0 + gy) % ney
                ge = gex + nex * (gey + ney * ez)
                for t2 in range(Nq):
                    for t1 in range(Nq):
                        nn = a_nb + Nq * (t1 + Nq * t2) if d == 0 else t1 + Nq * (a_nb + Nq * t2)
                        checked += 1
                        if not np.array_equal(Lf[sidx(gx, gy, ez), :, nn], G[ge, :, nn]):
                            errors += 1
    walls = [s for s in range(4) if nb[s] < 0]
    return dict(rank=rank, neighbours=nb, counts=cnt, errors=errors, checked=checked, walls=walls,
                interior_intact=bool(np.isfinite(Lf[[sidx(ex, ey, ez) for ez in range(nez) for ey in range(ny)
                                                     for ex in range(nx)]]).all()))


def main():
    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    out = []
    cases = [
        (dict(N=3, nex=5, ney=3, nez=2, Lx=5.0, Ly=3.0, Lz=2.0, periodic=(1, 1, 0)), 2, 1),
        (dict(N=3, nex=5, ney=3, nez=2, Lx=5.0, Ly=3.0, Lz=2.0, periodic=(0, 1, 0)), 2, 1),
        (dict(N=2, nex=3, ney=5, nez=3, Lx=3.0, Ly=5.0, Lz=3.0, periodic=(1, 1, 0)), 1, 2),
        (dict(N=4, nex=4, ney=4, nez=1, Lx=4.0, Ly=4.0, Lz=1.0, periodic=(1, 0, 0)), 1, 2),
        (dict(N=6, nex=4, ney=3, nez=2, Lx=4.0, Ly=3.0, Lz=2.0, periodic=(1, 1, 0)), 2, 1),
    ]
    for mesh, px, py in cases:
        out.append(dict(px=px, py=py, periodic=mesh["periodic"], **run_case(mesh, px, py, rank, world)))
        dist.barrier()
    with open(os.path.join(sys.argv[1], f"halo{rank}.json"), "w") as f:
        json.dump(out, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
