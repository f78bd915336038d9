"""Replicas with host-side dispatch across GPUs (one process per GPU).

Batched VQE parameter sets and served circuits are independent units (paper
Sec. III: the VQE loop asks for many energies; the serving workload is a
stream of unrelated circuits).  Over several GPUs each rank -- one process
per GPU, started by torchrun with RANK / WORLD_SIZE / LOCAL_RANK -- takes its
share of the units, runs them on its own GPU with its own streams and its own
memory budget, and the per-unit results are gathered on the host of rank 0.
Nothing is exchanged while units run: the only collectives are the final
gather of results (host objects) and the harness barriers, so the data path
has no collective at all.

Shares are deterministic functions of (unit count or request order, world
size, rank), so every unit is run exactly once and a result does not depend
on which rank ran it: a batched set's energies are those of the one-GPU run
bit for bit (each set is one CTA with no cross-set arithmetic).
"""
from __future__ import annotations

import numpy as np


def shard(n_units, world, rank):
    """Contiguous balanced share [lo, hi) of n_units for ``rank`` of ``world``
    (the first n_units % world ranks take one unit more)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_requests(requests, world, rank):
    """This rank's requests: the stream in arrival order, dealt round-robin
    (request k of the ordered stream goes to rank k % world), so every rank
    sees the same arrival rate and the same mix of sizes."""
    order = sorted(requests, key=lambda r: (r["arrival"], r["id"]))
    return order[rank::world]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def gather_to_root(obj, world, rank):
    """Every rank's ``obj`` in rank order on rank 0 (None elsewhere); with no
    process group (one process), [obj]."""
    dist = _dist()
    if dist is None or world == 1:
        return [obj]
    out = [None] * world if rank == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out


def run_batched(run_share, params, world=1, rank=0):
    """Energies of all parameter sets, computed in shares.

    run_share(lo, hi, params[lo:hi]) -> array (hi - lo, ne) runs one rank's
    sets on its GPU (for example a ``sim.Batch`` launch); the shares are
    gathered on rank 0 and concatenated in set order.  Returns the (nsets, ne)
    array on rank 0 and None on the other ranks."""
    params = np.asarray(params)
    lo, hi = shard(len(params), world, rank)
    local = np.asarray(run_share(lo, hi, params[lo:hi]))
    if local.shape[0] != hi - lo:
        raise ValueError("run_share returned the wrong number of sets")
    parts = gather_to_root((lo, hi, local), world, rank)
    if rank != 0:
        return None
    ne = max((p[2].shape[1] for p in parts if p[2].ndim == 2), default=0)
    out = np.empty((len(params), ne), dtype=local.dtype)
    covered = np.zeros(len(params), dtype=np.int64)
    for plo, phi, part in parts:
        out[plo:phi] = part
        covered[plo:phi] += 1
    if not np.all(covered == 1):
        raise RuntimeError("parameter sets not covered exactly once")
    return out


def serve_sharded(make_server, requests, world=1, rank=0, realtime=True):
    """Serve this rank's share of the stream on its own server.

    make_server() -> a ``serve.Server`` for this rank's GPU (its own executor,
    streams and admission budget).  Results (by request id) and each rank's
    budget figures are gathered on rank 0: returns (results, per-rank stats)
    there and (None, None) elsewhere."""
    mine = shard_requests(requests, world, rank)
    srv = make_server()
    res = srv.serve(mine, realtime=realtime)
    stats = dict(rank=rank, requests=len(mine), peak_bytes=srv.ledger.peak, budget=srv.ledger.budget,
                 wall=srv.wall)
    parts = gather_to_root((res, stats), world, rank)
    if rank != 0:
        return None, None
    merged = {}
    for part, _ in parts:
        for rid, r in part.items():
            if rid in merged:
                raise RuntimeError(f"request {rid} served twice")
            merged[rid] = r
    return merged, [s for _, s in parts]
