"""Continuous-batching serving loop over the C ABI.

Requests (see ``inputs.serve_requests``) arrive over time; each asks for
<Z_i> and the TFIM energy <H> of one circuit on a state vector or, with the
device noise model, on a density matrix.  The server keeps the GPU busy with
several requests at once:

* small state-vector requests (n <= ``batch_max_n``) are coalesced every
  ``tick`` seconds into one launch of the batched kernel (one CTA per
  request, whole state in shared memory);
* larger state-vector and all density-matrix requests are admitted against a
  byte budget (their state sizes) and run on ``slots`` CUDA streams by worker
  threads (the ABI calls release the Python GIL, so lowering, launches and
  reductions of different requests overlap);
* a request whose state alone exceeds the budget is rejected (EBUDGET), and
  one whose execution fails is reported with its error; neither stops the
  server.

Latency is completion time minus arrival time (host clock).  The executor
is pluggable so the admission logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import _lib as L


def state_bytes(req, dtype):
    if req["kind"] == "sv":
        return (16 if dtype == L.F64 else 8) << req["n"]
    return (8 if dtype == L.F64 else 4) << (2 * req["n"])


class Ledger:
    """Bytes in flight against a budget (admission control)."""

    def __init__(self, budget):
        self.budget = budget
        self.used = 0
        self.peak = 0
        self.cv = threading.Condition()

    def try_acquire(self, nbytes):
        with self.cv:
            if self.used + nbytes > self.budget:
                return False
            self.used += nbytes
            self.peak = max(self.peak, self.used)
            return True

    def release(self, nbytes):
        with self.cv:
            self.used -= nbytes
            self.cv.notify_all()


class GpuExecutor:
    """Runs requests through the CUDA library (one stream per worker).

    Lowered plans are cached by (kind, n, dtype, encoded gate bytes, noise
    parameters): repeated circuits skip lowering and the table upload."""

    def __init__(self, dtype=L.F32, plan_flags=0, cache_size=1024):
        import torch
        self.torch = torch
        self.dtype = dtype
        self.plan_flags = plan_flags
        self.cache = collections.OrderedDict()
        self.cache_size = cache_size
        self.seen = collections.OrderedDict()
        self.cache_lock = threading.Lock()
        self.hits = self.misses = 0

    def new_stream(self):
        return self.torch.cuda.Stream()

    def plan_for(self, req, arr, keep):
        """Cached plan for a circuit seen before, else None (one-shot path)."""
        from .sim import Plan
        if keep:  # caller matrices are referenced by address: not cacheable
            return None
        kind = L.SV if req["kind"] == "sv" else L.DM
        noise = req.get("noise")
        nkey = None
        if noise is not None:
            nkey = (np.asarray(noise["T1_us"]).tobytes(), np.asarray(noise["T2_us"]).tobytes(),
                    tuple(v for k, v in sorted(noise.items()) if k not in ("T1_us", "T2_us")))
        key = (kind, req["n"], self.dtype, self.plan_flags, arr.tobytes(), nkey)
        with self.cache_lock:
            p = self.cache.get(key)
            if p is not None:
                self.cache.move_to_end(key)
                self.hits += 1
                return p
            first = key not in self.seen
            if first:
                self.seen[key] = True
                while len(self.seen) > 8 * self.cache_size:
                    self.seen.popitem(last=False)
                self.misses += 1
                return None
        p = Plan(kind, req["n"], None, self.dtype, noise, self.plan_flags, encoded=arr)
        evicted = []
        with self.cache_lock:
            self.cache[key] = p
            while len(self.cache) > self.cache_size:
                evicted.append(self.cache.popitem(last=False)[1])
        del evicted  # rare: freeing plan tables synchronises the device
        return p

    def run_single(self, req, stream):
        from .sim import State
        kind = L.SV if req["kind"] == "sv" else L.DM
        ng = len(req["gates"])
        arr, keep = L.encode_gates_np(req["gates"])
        arr = arr[:ng]
        plan = self.plan_for(req, arr, keep)
        with State(kind, req["n"], self.dtype, stream=stream.cuda_stream) as st:
            if plan is not None:
                st.run(plan)
            else:  # first occurrence: one-shot lowering, tables released stream-ordered
                st.apply_encoded(arr, ng, req.get("noise"), self.plan_flags)
            z = st.expect(req["z_terms"], normalize=True)
            e = st.expect(req["h_terms"], sum=True, normalize=True)
        return dict(z=z, energy=e)

    def run_batch(self, reqs, stream):
        """Small SV requests as one batched launch: one template per request,
        energies = (<Z_0>..<Z_{n-1}>, <H>) via coefficient rows."""
        from .sim import Batch
        torch = self.torch
        templates, ne_max = [], 0
        for r in reqs:
            n, terms = r["n"], r["z_terms"] + r["h_terms"]
            nt = len(terms)
            coeffs = np.zeros((n + 1, nt))
            coeffs[np.arange(n), np.arange(n)] = 1.0
            coeffs[n, n:] = [t[2] for t in r["h_terms"]]
            templates.append(dict(n=n, gates=r["gates"], param_index=None, terms=terms, coeffs=coeffs))
            ne_max = max(ne_max, n + 1)
        with torch.cuda.stream(stream):
            b = Batch(templates, 0, self.dtype, stream=stream.cuda_stream)
            jt = torch.arange(len(reqs), dtype=torch.int32, device="cuda")
            out = torch.empty(len(reqs), ne_max, dtype=torch.float64, device="cuda")
            b.run(0, len(reqs), out.data_ptr(), ne_max, job_template_ptr=jt.data_ptr(), stream=stream.cuda_stream)
            res = out.cpu().numpy()  # synchronises the stream
            b.close()
        return [dict(z=res[i, :r["n"]].copy(), energy=float(res[i, r["n"]])) for i, r in enumerate(reqs)]


class Server:
    def __init__(self, executor, budget_bytes=150e9, slots=8, batch_max_n=12, batch_max=512, tick=0.002,
                 batch_streams=2, window=8, dtype=L.F32):
        self.ex = executor
        self.ledger = Ledger(budget_bytes)
        self.slots = slots
        self.batch_max_n = batch_max_n
        self.batch_max = batch_max
        self.tick = tick
        self.batch_streams = batch_streams
        self.window = window
        self.dtype = dtype

    # ------------------------------------------------------------ workers
    def _record(self, req, out=None, err=None, path=""):
        t = time.perf_counter()
        r = dict(id=req["id"], latency=t - (self.t0 + req["arrival"]), path=path, error=err, done_at=t - self.t0)
        if out:
            r.update(out)
        with self.lock:
            self.results[req["id"]] = r
            self.done += 1
            self.lock.notify_all()

    def _worker(self):
        stream = self.ex.new_stream()
        while True:
            with self.lock:
                req = None
                while req is None:
                    if self.closed and not self.large:
                        return
                    # first request in the head window whose state fits the budget
                    for i, r in enumerate(list(self.large)[:self.window]):
                        if self.ledger.try_acquire(state_bytes(r, self.dtype)):
                            req = r
                            del self.large[i]
                            break
                    if req is None:
                        self.lock.wait(0.01)
            nbytes = state_bytes(req, self.dtype)
            try:
                out = self.ex.run_single(req, stream)
                self._record(req, out, path="stream")
            except Exception as e:  # the failing request is reported; the server continues
                self._record(req, err=f"{type(e).__name__}: {e}", path="stream")
            finally:
                self.ledger.release(nbytes)
                with self.lock:
                    self.lock.notify_all()

    def _batcher(self):
        stream = self.ex.new_stream()
        while True:
            with self.lock:
                while not self.small and not self.closed:
                    self.lock.wait(self.tick)
                if self.closed and not self.small:
                    return
                take = []
                while self.small and len(take) < self.batch_max:
                    take.append(self.small.popleft())
            try:
                outs = self.ex.run_batch(take, stream)
                for r, o in zip(take, outs):
                    self._record(r, o, path="batch")
            except Exception as e:
                for r in take:
                    self._record(r, err=f"{type(e).__name__}: {e}", path="batch")
            time.sleep(self.tick)  # coalescing window for the next batch

    # ------------------------------------------------------------ driver
    def serve(self, requests, realtime=True):
        """Release requests at their arrival times; return results by id."""
        self.lock = threading.Condition()
        self.small, self.large = collections.deque(), collections.deque()
        self.results, self.done, self.closed = {}, 0, False
        threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(self.slots)]
        threads += [threading.Thread(target=self._batcher, daemon=True) for _ in range(self.batch_streams
                                                                                         if self.batch_max_n else 0)]
        self.t0 = time.perf_counter()
        for t in threads:
            t.start()
        for req in sorted(requests, key=lambda r: r["arrival"]):
            if realtime:
                delay = self.t0 + req["arrival"] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            if state_bytes(req, self.dtype) > self.ledger.budget:
                self._record(req, err="EBUDGET: state larger than the admission budget", path="rejected")
                continue
            with self.lock:
                if req["kind"] == "sv" and req["n"] <= self.batch_max_n:
                    self.small.append(req)
                else:
                    self.large.append(req)
                self.lock.notify_all()
        with self.lock:
            self.closed = True
            self.lock.notify_all()
            while self.done < len(requests):
                self.lock.wait(0.05)
        for t in threads:
            t.join(timeout=10)
        self.wall = time.perf_counter() - self.t0
        return self.results


def summarize(results, wall):
    lat = np.array([r["latency"] for r in results.values() if r["error"] is None])
    ok = len(lat)
    return dict(completed=ok, failed=len(results) - ok, circuits_per_s=ok / wall if wall > 0 else 0.0,
                p50_ms=float(np.percentile(lat, 50) * 1e3) if ok else None,
                p99_ms=float(np.percentile(lat, 99) * 1e3) if ok else None, wall_s=wall)
