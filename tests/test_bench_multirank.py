"""The benchmark's multi-rank path on CPU: two `gloo` ranks (one process each,
rendezvous on 127.0.0.1) exercise the barrier, the max-over-ranks time, the
whole-job value and the rank-0-only output of the reference arm."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), NWQ_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_init()
    dist.barrier()
    slowest = bench.reduce_max(1.5 + 2.0 * r, w)  # rank 1 is the slow one
    rate = bench.job_rate(100.0, w, slowest)
    out = io.StringIO()
    with redirect_stdout(out):
        rc = bench.run_reference(None, w, r) if r != 0 else 0  # rank 0's oracle run is not repeated here
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, slowest, rate, rc, out.getvalue()))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, slowest, rate, rc, out in res:
        assert w == 2 and slowest == pytest.approx(3.5)  # every rank sees the slowest time
        assert rate == pytest.approx(200.0 / 3.5)         # both ranks' units over that time
    assert res[1][4] == 0 and res[1][5] == ""           # the reference arm: rank 1 exits silently
