"""The multi-GPU path of the benchmark is replicas only (AxLocal has no
exchange step): each rank times its own replica and the job reports all
ranks' DOFs over the slowest rank's time.  Checked here with two gloo ranks
on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.reduce_max_ms(torch, 10.0 + 5.0 * rank, torch.device("cpu"))
    q.put((rank, ms, bench.whole_job_value(world, 1_000_000, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]  # both ranks see the slowest rank's time
    assert all(abs(r[2] - 2 * 1_000_000 / 15e-3 / 1e9) < 1e-12 for r in res)


def test_single_process_is_identity():
    import bench

    assert bench.reduce_max_ms(torch, 3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_value(1, 67_108_864, 3.0) == pytest.approx(22.369621333, rel=1e-9)
