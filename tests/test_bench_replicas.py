"""The multi-GPU path of the benchmark runs independent replicas (the method is
not sharded here): each rank times its own copy of the workload and the job's
rate is all ranks' element updates over the slowest rank's time.  Checked on the
CPU with two gloo ranks: the max-over-ranks reduction, the whole-job rate, and
that under torchrun only rank 0 runs and prints the reference arm."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, e2e = bench.max_over_ranks([10.0 + 5.0 * rank, 3.0 - rank], world)
    rate = bench.whole_job_rate(world, 1000, 20, ms)
    dist.destroy_process_group()
    out.put((rank, ms, e2e, rate))


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, rate in res:
        assert ms == 15.0 and e2e == 3.0                   # the slowest rank's times on every rank
        assert rate == pytest.approx(2 * 1000 * 20 / 15e-3)


def test_reference_arm_prints_on_rank_zero_only():
    """bench.py --impl reference under WORLD_SIZE = 2: rank 1 exits 0 without work
    or output (rank 0 would time the oracle; it is not run here)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
