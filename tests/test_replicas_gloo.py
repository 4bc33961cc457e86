"""Multi-rank aggregation of bench.py (replicas, one per rank) over a world-size-2 gloo group on CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2107_10423_gb300 import replicas
    ms = [1000.0, 1500.0][rank]            # rank 1 is slower
    units = [74.0, 74.0][rank]
    q.put((rank, replicas.aggregate(ms, units)))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, units, rate = out[r]
        assert ms == 1500.0 and units == 148.0
        assert abs(rate - 148.0 / 1.5) < 1e-9


def test_aggregate_single_process():
    from paper_2107_10423_gb300 import replicas
    assert replicas.aggregate(2000.0, 10.0) == (2000.0, 10.0, 5.0)
