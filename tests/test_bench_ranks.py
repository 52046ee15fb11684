"""The multi-GPU form of bench.py is replicas only: every rank solves its own
instance and the job time is the slowest rank's.  Its host logic runs here on
CPU with two gloo ranks (127.0.0.1)."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [3.0, 5.0][rank]
    slowest = bench.max_over_ranks(local_ms, world)
    out.put((rank, bench.replica_seed(rank), slowest, bench.job_ms_per_solve(slowest, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_instances():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [0, 1]            # one independent instance per rank
    assert all(g[2] == 5.0 for g in got)            # every rank sees the slowest time
    assert all(g[3] == 2.5 for g in got)            # two solves in 5 ms: 2.5 ms per solve


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25, 1) == 4.25 and bench.job_ms_per_solve(4.25, 1) == 4.25


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_oracle_pool_sample_on_host_cores():
    """The batched CPU baseline: a spawn process pool of oracle solves over
    a sample, extrapolated to the whole set by sum n^2."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1106_5694_gb300 import inputs
    ns = [30, 50, 70, 90]
    mats = [inputs.peer_shaped(n, 40 + k) for k, n in enumerate(ns)]
    objs = [int(oracle.dgs_parallel(m).objective) for m in mats]
    r = bench.oracle_pool_sample(lambda k: mats[k], ns, 2, objs)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["objectives_equal_to_gpu"]
    assert r["value"] > 0 and "(2 of 4)" in r["sample"]  # instances 0 and 2
    wrong = list(objs)
    wrong[2] += 1
    assert not bench.oracle_pool_sample(lambda k: mats[k], ns, 2, wrong)["objectives_equal_to_gpu"]
