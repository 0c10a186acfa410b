"""The multi-GPU path is replicas only: every rank convolves its own densities, the job's time is
the slowest rank's, and throughput sums the ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 100.0 + 50.0 * rank          # rank 1 is slower
    mx = bench.max_over_ranks(ws, ms, device="cpu")
    rate = bench.job_throughput(ws, 80, mx)
    bench.barrier(ws)
    q.put((rank, mx, rate))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate in res:
        assert mx == 150.0
        assert rate == pytest.approx(2 * 80 / 0.150)
