"""The benchmark's multi-rank path (replicas: one transform per GPU, the job
time is the slowest rank's) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _child(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], torch.device("cpu"))
        out.put((rank, t, bench.job_rate(world, 2, 1 << 30, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [95.0, 101.5]
    port = _free_port()
    procs = [ctx.Process(target=_child, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for rank, t, rate in res:
        assert t == max(times)
        assert rate == pytest.approx(2 * 2 * bench.flops(1 << 30) / (max(times) * 1e-3) / 1e9)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
