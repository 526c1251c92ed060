"""The multi-GPU path of the benchmark is replicas only: every rank runs an
independent controller and the job's throughput is all ranks' sample-steps
over the slowest rank's time.  These CPU tests run that reduction over two
gloo ranks (127.0.0.1) and in a single process."""
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        seconds = [2.0, 3.0, 2.5, 1.0][rank]          # rank 1 is the slowest
        thr, t = bench.replica_throughput(1000, seconds)
        a, b = bench.slowest_rank(float(rank), 10.0 - rank)
        q.put((rank, thr, t, a, b))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_replica_throughput_over_gloo_ranks(ws):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    try:
        got = [q.get(timeout=120) for _ in range(ws)]
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, thr, t, a, b in got:
        assert t == 3.0                              # the slowest rank's time on every rank
        assert thr == pytest.approx(1000 * ws / 3.0)  # every rank's units over it
        assert (a, b) == (float(ws - 1), 10.0)       # element-wise maximum


def test_replica_throughput_single_process():
    import bench
    thr, t = bench.replica_throughput(1000, 2.0)
    assert (thr, t) == (500.0, 2.0)
    assert bench.slowest_rank(1.5, 2.5) == (1.5, 2.5)
