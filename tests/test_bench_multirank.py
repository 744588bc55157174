"""The bench's multi-rank host path on CPU: two gloo ranks report different step times, every
rank sees the slowest, and the whole-job throughput counts both replicas' work in that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench.slowest_rank_ms(10.0 * (rank + 1), ws, "cpu")
    out.put((rank, ms, bench.whole_job_tflops(2.0e12, ms, ws)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    assert [r for r, _, _ in res] == [0, 1]
    for _, ms, tf in res:
        assert ms == 20.0
        assert tf == pytest.approx(2 * 2.0e12 / 0.020 / 1e12)


def test_single_rank_is_unchanged():
    import bench
    assert bench.slowest_rank_ms(7.5, 1, "cpu") == 7.5
    assert bench.whole_job_tflops(1e12, 1000.0, 1) == pytest.approx(1.0)
