"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): the
slowest rank's time is taken (max over ranks), the whole-job value counts
every rank's replica, and the reference arm runs on rank 0 alone.  No GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank                 # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms_local)
    value = bench.job_throughput(1000, 2, 50, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms_max, value))


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in got:
        assert ms_max == 15.0                    # every rank sees the slowest rank's time
        assert abs(value - 1000 * 2 * 50 * world / 15e-3 / 1e6) < 1e-9


def test_max_over_ranks_without_a_group_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm prints from rank 0; another rank
    exits 0 at once without work and prints nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_rank_zero():
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys (one bounded oracle step on the host cores)."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "config", "cpu_baseline", "e2e", "higher_is_better"):
        assert k in line
