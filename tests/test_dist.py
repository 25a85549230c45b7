"""Multi-rank aggregation of bench.py on CPU: two gloo ranks, max-over-ranks timing and the
weak-scaling whole-job rate (no GPU needed)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    my_ms = [12.5, 40.0][rank]
    slowest = bench.max_over_ranks(my_ms, dist, "cpu")
    dist.barrier()
    q.put((rank, slowest, bench.weak_scaling_rate(1e6, world, slowest)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
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
    assert [o[1] for o in out] == [40.0, 40.0]
    assert out[0][2] == pytest.approx(2e6 / 0.040)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_scaling_rate(100.0, 1, 1000.0) == pytest.approx(100.0)
