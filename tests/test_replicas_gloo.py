"""The multi-GPU path of bench.py is replicas: each rank compresses its own stream and
the ranks meet only for the barrier and the max-over-ranks time.  Exercised here with
two gloo ranks on the CPU (no GPU): the aggregation every rank computes, the barrier,
and the per-rank seeds."""

import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import datetime
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    import bench
    ms_local = [120.0, 150.0][rank]          # device-event time of this rank's K steps
    host_local = [0.100, 0.130][rank]        # host-clock time of the same steps
    value, ms_total = bench.replica_value(world, 100, ms_local, host_local)
    mx = bench.max_over_ranks(float(10 * rank + 1), world)
    bench.barrier(world)
    queue.put((rank, value, ms_total, mx, bench.replica_seed("reactive", rank), bench.replica_seed("channel", rank)))
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, value, ms_total, mx, seed_r, seed_c = queue.get(timeout=120)
        got[rank] = (value, ms_total, mx, seed_r, seed_c)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the slowest rank sets the time (150 ms, larger than either host clock); every
    # rank reports the same whole-job figure: 2 ranks x 100 steps / 0.150 s
    for rank in (0, 1):
        value, ms_total, mx, _, _ = got[rank]
        assert ms_total == 150.0
        assert abs(value - 2 * 100 / 0.150) < 1e-9
        assert mx == 11.0
    # rank 0 keeps the named configuration's seed; the other replica gets its own stream
    assert got[0][3] is None and got[0][4] is None
    assert got[1][3] == 1012 and got[1][4] == 1014
