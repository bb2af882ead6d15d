"""The multi-rank logic of bench.py (replicas only: a barrier and the maximum
of the per-rank timed region, no data-path collective) with the gloo backend,
world size 2, on CPU."""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench

    r, w, lr = bench.dist_env()
    dist = bench.init_dist(w, lr)
    mx = bench.max_over_ranks(dist, 10.0 * (r + 1))
    bench.barrier(dist)
    q.put((r, w, mx))
    dist.destroy_process_group()


def test_two_rank_max_and_barrier_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2, 20.0), (1, 2, 20.0)]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.init_dist(1, 0) is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
