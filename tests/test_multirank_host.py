"""The benchmark's multi-rank logic on CPU with the gloo backend (world size 2):
every rank gets its own workload seed (weak scaling, no data-path collective),
the reported time is the maximum over ranks, the throughput is the units of
all ranks over that time, and the reference arm prints on rank 0 only."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    # unequal work per rank: 1,000 and 3,000 units in 10 and 15 ms -> 4,000 units / 15 ms
    v = bench.job_throughput(1000.0 + 2000.0 * rank, 10.0 + 5.0 * rank, "cpu")
    out.put((rank, t, bench.rank_seed(rank), v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_per_rank_seeds_gloo():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] != res[1][2]
    for r in res:
        assert abs(r[3] - 4000.0 / 0.015) <= 1e-6 * r[3]


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5


def test_single_process_throughput():
    import bench
    assert abs(bench.job_throughput(560000.0, 500.0, "cpu") - 1.12e6) < 1e-3


def test_reference_arm_prints_on_rank0_only():
    """Under torchrun every rank runs bench.py --impl reference; only rank 0
    runs the oracle and prints the line, the others exit 0 without work."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
