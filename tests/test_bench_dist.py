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


def _oracle_worker(rank, world, port, q):
    """One rank of the sample-sharded path: the replicated tiny graph, this rank's own
    samples, the rank's partial sum from the oracle, then the one exchange (an FP64
    all-reduce of sum and count) giving the mean over both ranks' samples."""
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    base = tiny(num_samples=700 + 300 * r)          # uneven shards
    mine = tiny(seed=bench.rank_seed(0, r), num_samples=700 + 300 * r)
    R, _ = oracle.evaluate(base.graph, mine.samples.eps, mine.samples.beta, mine.samples.t)
    mean = bench.combine_means(oracle.neumaier_sum(R), R.size, w)
    q.put((r, mean))
    dist.destroy_process_group()


def test_two_rank_oracle_means_combine_over_all_samples():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    base = tiny(num_samples=700)
    ts = [tiny(seed=bench.rank_seed(0, r), num_samples=700 + 300 * r).samples for r in range(2)]
    R_all = np.concatenate([oracle.evaluate(base.graph, s.eps, s.beta, s.t)[0] for s in ts])
    want = oracle.neumaier_mean(R_all)
    _, A_all = oracle.evaluate(base.graph, ts[0].eps, ts[0].beta, np.concatenate([s.t for s in ts]))
    for _, m in res:
        assert abs(m - want) <= 1e-13 * float(np.mean(A_all))


def test_bench_starts_its_own_ranks_for_several_gpus():
    """bench.py --gpus 2 without a torchrun environment launches two ranks itself;
    with the reference arm only rank 0 works and prints the one JSON line."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR",
                                                             "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--impl", "reference",
                        "--workload", "tiny", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


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


def test_profiled_traffic_scales_with_samples_and_checks_the_schedule():
    """The committed ncu figure is per launch at the profiled sample count; other sample
    counts scale it, and a launch on another schedule gets no figure."""
    import json
    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")) as f:
        d = json.load(f)
    for tag, v in d.items():
        full = bench.profiled_traffic(tag, v["samples"], v["schedule"], v["layout"])
        assert full == v["bytes_per_launch"]
        assert bench.profiled_traffic(tag, v["samples"] // 4, v["schedule"], v["layout"]) == full / 4
        assert bench.profiled_traffic(tag, v["samples"], 3 - v["schedule"], v["layout"]) is None
        assert bench.profiled_traffic(tag, v["samples"], v["schedule"], v["layout"] + 1) is None
    assert bench.profiled_traffic("walk_count_nothing", 1, 1, 1) is None


def test_profiled_traffic_entries_name_their_ncu_summaries():
    """Every traffic figure the bench may report names the committed ncu summary it was
    read from, and that summary exists and gives the same per-capture bytes."""
    import json
    import re
    root = os.path.dirname(bench.__file__)
    with open(os.path.join(root, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for tag, v in d.items():
        m = re.search(r"profiles/([\w.]+\.md)", v["source"])
        assert m, tag
        path = os.path.join(root, "profiles", m.group(1))
        assert os.path.exists(path), (tag, path)
        # the capture's read + write bytes (GB, 3 decimals) appear in the summary
        gb = re.search(r"\(([\d.]+) \+ ([\d.]+) = ([\d.]+) GB\)", v["source"])
        assert gb, tag
        with open(path) as f:
            text = f.read()
        assert f"{gb.group(1)} + {gb.group(2)} = {gb.group(3)} GB" in text, tag


def test_serving_oracle_check_flags_a_wrong_mean():
    """The serving line's check: requests whose served means equal the oracle's pass;
    one served mean moved by 1e-3 of the mean of sum |paths| is flagged.  Counter-drawn
    times (the resident server's generator) only, so no device is needed."""
    import oracle
    from paper_2501_00675_gb300.serve import Request, RequestSpec
    from workloads import counter_times
    w = tiny(seed=5)
    wpool = [(w.graph, w.samples.eps)]
    reqs, scale = [], []
    for q, S in enumerate((40, 130, 7)):
        spec = RequestSpec(0, S, 1000 + q)
        R, A = oracle.evaluate(w.graph, w.samples.eps, 10.0, counter_times(spec.seed, 0, S, w.graph.num_times, 10.0))
        r = Request(spec=spec, need_bytes=0, t_submit=0.0, rid=q, status="done", mean=oracle.neumaier_mean(R))
        reqs.append(r)
        scale.append(float(np.mean(A)))
    reqs.append(Request(spec=RequestSpec(0, 50, 9), need_bytes=0, t_submit=0.0, rid=9, status="shed"))
    ok = bench.serving_oracle_check(None, reqs, wpool, 10.0, 1, counter=True)
    assert ok["within_tolerance"] and ok["requests_checked"] == 3
    assert ok["max_mean_err_over_mean_abs_path_sum"] == 0.0
    reqs[1].mean += 1e-3 * scale[1]
    bad = bench.serving_oracle_check(None, reqs, wpool, 10.0, 1, counter=True)
    assert not bad["within_tolerance"]
    assert abs(bad["max_mean_err_over_mean_abs_path_sum"] - 1e-3) < 1e-9


def test_batched_oracle_check_flags_a_wrong_sample():
    """The batched line's check on host arrays: the oracle's own values pass (and the
    path counts in count mode); one sample moved by 1e-3 of its sum |paths| is flagged."""
    import oracle
    wls = [tiny(seed=11, num_samples=40), tiny(seed=12, num_samples=25)]
    got, scale = [], []
    for w in wls:
        R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:16])
        got.append(R.copy())
        scale.append(A)
    ok = bench.batched_oracle_check(wls, got, 1)
    assert ok["within_tolerance"] and ok["samples_checked"] == 32 and ok["max_err_over_abs_path_sum"] == 0.0
    got[1][3] += 1e-3 * scale[1][3]
    bad = bench.batched_oracle_check(wls, got, 1)
    assert not bad["within_tolerance"] and abs(bad["max_err_over_abs_path_sum"] - 1e-3) < 1e-9
    counts = [np.full(8, oracle.count_paths(w.graph)[0], dtype=np.int64) for w in wls]
    assert bench.batched_oracle_check(wls, counts, 2)["bit_exact"]
    counts[0][2] += 1
    assert not bench.batched_oracle_check(wls, counts, 2)["bit_exact"]


def test_batched_reference_arm_times_the_oracle_on_the_same_mix():
    args = bench.parse_args(["--impl", "reference", "--workload", "batched", "--num-graphs", "3",
                             "--steps", "1", "--warmup", "0", "--reference-seconds", "1"])
    assert bench.run_reference_batched(args, rank=1, world=2) is None
    line = bench.run_reference_batched(args, rank=0, world=1)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == bench.batched_desc(3)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
