"""Host-side logic of the multi-GPU benchmark path, run as two gloo ranks on CPU:
weak scaling gives every rank its own samples of the same graph, the timed region
is the maximum over ranks, and the means combine over all ranks' samples."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from workloads import tiny


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    m = bench.max_over_ranks(float(10 * (rank + 1)), w)
    wl = tiny(seed=bench.rank_seed(0, r), num_samples=8)
    mean = bench.combine_means([3.0, 5.0][r], [2, 6][r], w)   # (3 + 5) / (2 + 6)
    bench.barrier(w)
    q.put((r, m, wl.samples.t.sum(), wl.graph.edges.sum(), mean))
    dist.destroy_process_group()


def test_two_rank_max_and_sample_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]          # max over ranks seen by both
    assert [r[4] for r in res] == [1.0, 1.0]            # mean over both ranks' samples
    assert res[0][2] != res[1][2]                        # rank samples differ (own seeds)
    assert bench.rank_seed(1, 0) == 1                    # rank 0 keeps the workload's own samples


def test_reference_arm_on_other_ranks_does_no_work():
    args = bench.parse_args(["--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args, rank=1, world=2) is None
    line = bench.run_reference(args, rank=0, world=1)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
