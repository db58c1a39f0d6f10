"""bench.py at N > 1 runs independent replicas, one per rank (the path has no
data-path exchange).  Its whole-job numbers are the slowest rank's time and
the sum of the ranks' updates; checked here with two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sec, upd = bench.replica_totals(1.0 + rank, 10.0 * (rank + 1), "cpu")
    q.put((rank, sec, upd))
    dist.destroy_process_group()


def test_two_replicas_max_time_sum_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, sec, upd in got:
        assert sec == 2.0 and upd == 30.0
