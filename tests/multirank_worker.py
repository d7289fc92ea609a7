"""Worker for the two-rank CPU test of the bench's rank logic (gloo): each
rank reports a different time, and every rank must see the maximum and the
same whole-job rate.  Launched by tests/test_multirank_cpu.py under
torch.distributed.run."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import bench  # noqa: E402


def main():
    world, rank, local = bench.dist_setup()
    torch.distributed.init_process_group("gloo")
    ms = 100.0 + 50.0 * rank
    worst = bench.max_over_ranks(ms, world, torch, "cpu")
    rate = bench.whole_job_rate(1000, world, 3, worst)
    torch.distributed.barrier()
    # one file per rank: the ranks' stdout streams interleave
    with open(os.path.join(sys.argv[1], f"rank{rank}.json"), "w") as f:
        json.dump(dict(rank=rank, world=world, local=local, worst=worst, rate=rate), f)
    torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
