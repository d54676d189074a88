"""Multi-GPU is replicas only: N ranks run independent copies and the job time
is the maximum over ranks.  The aggregation runs here as 2 gloo ranks on CPU."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v, t = bench.replica_value(units=1000.0, ms_local=10.0 * (rank + 1), world=world, device="cpu")
    q.put((rank, v, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_takes_the_slowest_rank():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, v, t in out:
        assert t == 20.0                      # max over ranks
        assert abs(v - 2 * 1000.0 / 0.020) < 1e-6
