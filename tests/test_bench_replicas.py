"""The multi-rank path of bench.py on CPU: two gloo ranks aggregate their
replica timings into one whole-job throughput (max time over ranks, units of
all ranks), and the reference arm does its work on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, ms: list, ssu: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, bench.replica_throughput(ms[rank], ssu, "cpu")))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_all_units():
    world, ssu = 2, 50_331_648 * 10
    ms = [21.5, 23.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms, ssu, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        ms_max, value = res[r]
        assert ms_max == max(ms)
        assert value == pytest.approx(world * ssu / (max(ms) * 1e-3) / 1e9, rel=1e-15)


def test_single_process_is_one_replica():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.replica_throughput(4.0, 1_000_000, "cpu")
    assert ms_max == 4.0 and value == pytest.approx(1_000_000 / 4e-3 / 1e9)


def test_reference_arm_on_a_nonzero_rank_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
