"""The multi-process plumbing of bench.py on CPU: two gloo ranks (world size
2, 127.0.0.1) go through its process-group setup, barrier and max-over-ranks
timing, and the reference arm's non-zero rank exits without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        impl = "reference"   # gloo: no GPU here
        gpus = world
    w, r, local, pg = bench.dist_setup(Args)
    try:
        bench.barrier(pg)
        m = bench.max_over_ranks(pg, 1.5 + rank)
        # the reference arm: ranks other than 0 exit 0 without work
        rc = bench.run_reference(Args, w, r, pg) if r != 0 else 0
        out.put((r, w, m, rc))
    finally:
        pg.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5, 0), (1, 2, 2.5, 0)]
