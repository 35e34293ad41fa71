"""The benchmark's multi-replica logic on CPU: two gloo ranks, each timing
its own replica; the job time is the slowest rank's and the throughput sums
the ranks' work (no collective touches the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms_local = 10.0 + 5.0 * rank            # rank 1 is the slower replica
    ms = bench.reduce_max(ms_local, ws, device="cpu")
    rate = bench.aggregate_rate(1000.0, ms, ws)
    wsr, rnk, local = bench._dist()
    q.put((rank, ms, rate, wsr, rnk, local))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, wsr, rnk, local in out:
        assert ms == 15.0                     # max over ranks
        assert rate == pytest.approx(2 * 1000.0 / 0.015)
        assert (wsr, rnk, local) == (2, rank, rank)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate_rate(10.0, 2.0, 1) == pytest.approx(5000.0)
