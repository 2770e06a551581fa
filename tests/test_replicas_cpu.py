"""The N > 1 path of bench.py runs independent replicas; only the elapsed time
(max) and the unit count (sum) are reduced. Checked with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    # rank r took (r + 1) * 100 ms for 3 sweeps
    v, ms = bench.replica_throughput((rank + 1) * 100.0, 3, "cpu")
    q.put((rank, v, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, v, ms in res:
        assert ms == 200.0                      # slowest rank
        assert abs(v - 6 / 0.2) < 1e-9         # 2 x 3 sweeps in 0.2 s
