"""Per-GPU dispatch of independent units (batched VQE sets, served circuits)
on CPU: two `gloo` ranks (one process each, rendezvous on 127.0.0.1), each
with a fake per-device executor, against the one-rank run.  Checked: every
set and every request runs exactly once, the merged results equal the
one-rank results bit for bit, and each rank's admission budget holds."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import dispatch, inputs
from paper_2401_06861_gb300.serve import Server, state_bytes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUDGET = 2 * state_bytes(dict(kind="sv", n=18), L.F32)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def fake_energies(lo, hi, params):
    """Stand-in for one GPU's batched launch: energies of each set from its
    parameters only (three h values), plus the set's global index as a
    fourth column so the gather's placement can be checked."""
    p = np.asarray(params, np.float64)
    e = np.stack([np.cos(p).sum(axis=1) * h for h in (0.5, 1.0, 2.0)], axis=1)
    return np.concatenate([e, np.arange(lo, hi, dtype=np.float64)[:, None]], axis=1)


def make_server():
    from tests.test_serve_host import FakeExecutor
    ex = FakeExecutor(delay=0.001)
    srv = Server(ex, budget_bytes=BUDGET, slots=3, batch_max_n=10)
    ex.server = srv
    return srv


def workloads():
    params = inputs.hea_params(6, 2, 101, seed=7)
    reqs = inputs.serve_requests(rate=1500, duration=0.08, seed=11, sv_n=(8, 18), dm_n=(6, 8))
    return params, reqs


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    params, reqs = workloads()
    energies = dispatch.run_batched(fake_energies, params, ws, rank)
    res, stats = dispatch.serve_sharded(make_server, reqs, ws, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, energies, None if res is None else {k: (v["energy"], v["error"]) for k, v in res.items()}, stats))


def test_shards_cover_every_unit_once():
    for n in (0, 1, 7, 64, 101):
        for ws in (1, 2, 3, 8):
            spans = [dispatch.shard(n, ws, r) for r in range(ws)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    _, reqs = workloads()
    got = sorted(r["id"] for k in range(3) for r in dispatch.shard_requests(reqs, 3, k))
    assert got == sorted(r["id"] for r in reqs)


def test_two_gloo_ranks_batched_sets_and_serving():
    import torch.multiprocessing as mp
    params, reqs = workloads()
    one_e = dispatch.run_batched(fake_energies, params)
    one_res, one_stats = dispatch.serve_sharded(make_server, reqs)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, e0, res0, stats0), (_, e1, res1, stats1) = out
    assert e1 is None and res1 is None and stats1 is None      # results live on rank 0 only
    assert np.array_equal(e0, one_e)                           # bitwise equal to the one-rank run
    assert np.array_equal(e0[:, 3], np.arange(len(params)))    # each set placed once, in order
    assert sorted(res0) == sorted(r["id"] for r in reqs)       # each request served exactly once
    assert all(err is None for _, err in res0.values())
    assert {k: v["energy"] for k, v in one_res.items()} == {k: e for k, (e, _) in res0.items()}
    assert [s["rank"] for s in stats0] == [0, 1] and sum(s["requests"] for s in stats0) == len(reqs)
    for s in stats0:                                           # every rank kept its own budget
        assert s["budget"] == BUDGET and 0 < s["peak_bytes"] <= BUDGET
    assert one_stats[0]["peak_bytes"] <= BUDGET
