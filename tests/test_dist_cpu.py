"""The bench's multi-rank logic on CPU: two gloo ranks (one process per GPU in a real run).

bench.py runs one independent shell per rank (replicas, no collective on the data
path); the ranks only agree on the time, which is the slowest rank's, and only rank 0
prints.  This test runs that agreement and the reference arm's rank gate with gloo."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_setup('gloo')
    assert (r, w, local) == (rank, ws, rank)
    m = bench.max_over_ranks(10.0 + 3 * rank, 'cpu')
    # the reference arm runs on rank 0 only: the other ranks return at once
    gated = rank != 0 and bench.reference_arm(None, rank, ws) is None
    out.put((rank, m, gated))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1] == 13.0
    assert res[1][2]
