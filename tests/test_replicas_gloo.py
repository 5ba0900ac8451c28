"""Host logic of the benchmark's multi-GPU mode ("replicas only": every rank
subtracts its own CCD pairs, no data-path collective) on two CPU ranks over
gloo: each rank draws an independent pair from the same recipe, and the
timing reduction takes the maximum over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    args = argparse.Namespace(batch=1, rows=64)
    pairs = bench.load_pairs(args, rank)
    checksum = float(pairs[0]["R"].astype("float64").sum())
    t = bench._max_over_ranks(dist, torch.device("cpu"), 1.0 + rank)
    q.put((rank, pairs[0]["R"].shape, checksum, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_draw_independent_pairs_and_reduce_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, shp0, c0, t0), (r1, shp1, c1, t1) = out
    assert shp0 == shp1 == (64, 2048)
    assert c0 != c1                      # independent pairs per rank
    assert t0 == t1 == 2.0               # max over ranks
