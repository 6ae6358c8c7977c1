"""The N > 1 path of bench.py (independent replicas, one per rank) on the CPU:
two gloo ranks rendezvous on 127.0.0.1, pass the barrier and agree on the
maximum of their step times -- the timing rule the benchmark applies."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "CUDA_VISIBLE_DEVICES": ""})
    import torch.distributed as dist

    import bench

    ws, r, local = bench.dist_setup()
    assert (ws, r) == (world, rank)
    bench.barrier(ws)
    m = bench.allreduce_max(10.0 + rank * 5.0, ws)
    q.put((rank, m, dist.get_backend()))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_replicas_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(90)
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert [p.exitcode for p in ps] == [0, 0]
    assert res == [(0, 15.0, "gloo"), (1, 15.0, "gloo")]
