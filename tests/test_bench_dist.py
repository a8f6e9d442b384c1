"""The benchmark's multi-rank path on CPU: two gloo ranks agree on the job
time (max over ranks) and rank 0 reports the whole-job rate (weak scaling:
each rank runs its own stream, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [120.0, 150.0][rank]           # rank 1 is the slow one
    dist.barrier()
    t = bench.job_time_ms(local, ws, torch.device("cpu"))
    rate = bench.whole_job_rate(30, ws, t)
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_rank_job_time_is_the_max_and_rate_counts_every_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in out:
        assert t == 150.0                          # both ranks see the slowest rank's time
        assert abs(rate - 2 * 30 / 0.150) < 1e-9   # 60 frames in 150 ms


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_time_ms(42.0, 1, None) == 42.0
    assert bench.whole_job_rate(10, 1, 20.0) == 500.0
