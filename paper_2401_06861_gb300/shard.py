"""One state vector sharded over G = 2^g GPUs by its top qubits.

The paper runs SV-Sim on multi-node, multi-GPU systems for states that do not
fit one device (Sec. II; Sec. V).  Here the 2^n amplitudes are split by the
top g bits of the *physical* index: slice r (rank r) holds the 2^L amplitudes
(L = n - g) whose top g physical bits equal r.  A qubit map assigns each
logical qubit a physical bit; qubits on bits below L are local, the g
others are global (they select the slice).

* A gate whose qubits are all local runs on every slice as a gate of an
  L-qubit state vector (the library's sweep kernels, unchanged).
* A gate on a global qubit first swaps that qubit with a local one: with
  global bit L + j and local bit l, rank r keeps the half of its slice whose
  bit l equals bit j of r and exchanges the other half with rank r ^ 2^j
  (one send and one receive of 2^(L-1) amplitudes; with l = L - 1 the half
  is contiguous).  The received half is staged in local memory and copied
  into place; the two qubits' physical bits trade places in the map.
* <P> of a Pauli string whose X support is local is a sum over the slices of
  local sums, the global Z bits contributing the sign (-1)^{|r & z_glob|};
  strings with global X support first swap those qubits in (X support on at
  most L qubits; wider strings are refused).  One all-reduce of the per-term
  sums ends the evaluation.

Slice storage and local arithmetic come from a backend (``GpuSlices``: the
library on the rank's GPU; the tests use the CPU oracle on each slice), and
the exchange from a transport: ``DistTransport`` (torch.distributed point to
point, NCCL between GPUs or gloo on CPU, one slice per process) or
``LocalTransport`` (all slices in one process, halves swapped by copies).
"""
from __future__ import annotations

import numpy as np


class QubitMap:
    """Logical qubit -> physical bit (a permutation of 0..n-1)."""

    def __init__(self, n):
        self.n = n
        self.phys = list(range(n))

    def logical_at(self, bit):
        return self.phys.index(bit)

    def swap_bits(self, a, b):
        qa, qb = self.logical_at(a), self.logical_at(b)
        self.phys[qa], self.phys[qb] = b, a

    def mask(self, m):
        """A logical bit mask as a physical one."""
        out = 0
        for q in range(self.n):
            if (m >> q) & 1:
                out |= 1 << self.phys[q]
        return out


def half_view(t, L, l, c):
    """The 2^(L-1) elements of a 2^L slice whose bit l is c, as a view."""
    return t.view(1 << (L - 1 - l), 2, 1 << l)[:, c, :]


class LocalTransport:
    """All slices in this process: a pairwise exchange swaps two halves."""

    def exchange(self, sv, j, l):
        L = sv.L
        for r in sv.ranks:
            p = r ^ (1 << j)
            if p < r:
                continue
            a = half_view(sv.tensor(r), L, l, 1 - ((r >> j) & 1))
            b = half_view(sv.tensor(p), L, l, 1 - ((p >> j) & 1))
            stage = a.clone()  # staged, then both halves written
            a.copy_(b)
            b.copy_(stage)

    def allreduce(self, sv, v):
        return v

    def gather(self, sv, parts):
        return parts


class DistTransport:
    """One slice per process: halves exchanged with torch.distributed point to
    point (isend / irecv), received into a staging buffer, then copied in."""

    def __init__(self, chunk=1 << 26):
        import torch.distributed as dist
        self.dist = dist
        self.chunk = chunk  # amplitudes per message (bounds the staging buffer)

    def exchange(self, sv, j, l):
        (r,) = sv.ranks
        p = r ^ (1 << j)
        mine = half_view(sv.tensor(r), sv.L, l, 1 - ((r >> j) & 1))
        if mine.is_contiguous():  # l = L - 1: one contiguous half, in chunks
            flat = mine.reshape(-1)
            for a in range(0, flat.numel(), self.chunk):
                b = min(flat.numel(), a + self.chunk)
                self._sendrecv(flat[a:b].clone(), flat[a:b], p)
        else:  # a strided half: packed, exchanged, unpacked
            packed = mine.contiguous().reshape(-1)
            self._sendrecv(packed, None, p, into=mine)

    def _sendrecv(self, send, dst, peer, into=None):
        import torch
        recv = torch.empty_like(send)  # staging buffer in local memory
        ops = [self.dist.P2POp(self.dist.isend, send, peer), self.dist.P2POp(self.dist.irecv, recv, peer)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()
        if into is not None:
            into.copy_(recv.view_as(into))
        else:
            dst.copy_(recv)

    def allreduce(self, sv, v):
        import torch
        t = torch.as_tensor(np.asarray(v, np.float64), device=sv.comm_device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()

    def gather(self, sv, parts):
        out = [None] * sv.world
        self.dist.all_gather_object(out, parts[0])
        return out


class ShardedSV:
    """An n-qubit state vector over 2^g slices (see the module notes).

    ranks: the slice indices this process holds (all of them with
    LocalTransport, its own rank with DistTransport).  backend: slice storage
    and local arithmetic (zeros / unit / tensor / apply / expect / numpy)."""

    def __init__(self, n, g, backend, transport, ranks, comm_device="cpu"):
        if not 0 <= g < n:
            raise ValueError("need 0 <= g < n")
        self.n, self.g, self.L = n, g, n - g
        self.world = 1 << g
        self.backend, self.transport = backend, transport
        self.ranks = sorted(ranks)
        self.comm_device = comm_device
        self.map = QubitMap(n)
        self.slices = {r: (backend.unit(self.L) if r == 0 else backend.zeros(self.L)) for r in self.ranks}
        self.exchanges = 0

    def tensor(self, r):
        return self.backend.tensor(self.slices[r])

    # ------------------------------------------------------------ layout
    def _make_local(self, qubits, keep=()):
        """Swap every global qubit of ``qubits`` with a local one (the highest
        local bit whose qubit is not in ``keep``)."""
        keep = set(keep) | set(qubits)
        for q in qubits:
            bit = self.map.phys[q]
            if bit < self.L:
                continue
            victims = [b for b in range(self.L - 1, -1, -1) if self.map.logical_at(b) not in keep]
            if not victims:
                raise ValueError("not enough local qubits for this gate or term")
            l = victims[0]
            self.transport.exchange(self, bit - self.L, l)
            self.map.swap_bits(bit, l)
            self.exchanges += 1

    # ------------------------------------------------------------ circuits
    def apply(self, gates):
        """Apply gates (name, logical qubits, params), grouping runs of gates
        whose qubits are local into one call per slice."""
        run = []
        for name, qs, prm in gates:
            if any(self.map.phys[q] >= self.L for q in qs):
                self._flush(run)
                run = []
                self._make_local(qs)
            run.append((name, tuple(self.map.phys[q] for q in qs), prm))
        self._flush(run)

    def _flush(self, run):
        if run:
            for r in self.ranks:
                self.backend.apply(self.slices[r], run)

    # ------------------------------------------------------------ measurement
    def expect(self, terms):
        """Per-term <P> (coefficients not applied), summed over all slices.
        Terms are evaluated in order, in batches under one qubit map; a term
        with X support on global qubits first swaps them in."""
        vals = np.zeros(len(terms))
        full = (1 << self.n) - 1
        lowm = (1 << self.L) - 1
        batch = []  # (k, local x, local z, global z) under the current map

        def flush():
            if not batch:
                return
            loc = [(lx, lz, 1.0) for _, lx, lz, _ in batch]
            for r in self.ranks:
                v = self.backend.expect(self.slices[r], loc)
                for (k, _, _, gz), vk in zip(batch, v):
                    vals[k] += -vk if bin(r & gz).count("1") & 1 else vk
            batch.clear()

        for k, (x, z, _) in enumerate(terms):
            x, z = x & full, z & full
            xs = [q for q in range(self.n) if (x >> q) & 1 and self.map.phys[q] >= self.L]
            if xs:
                if bin(x).count("1") > self.L:
                    raise ValueError("a Pauli string with X support on more than n - g qubits needs more local "
                                     "qubits than a slice has")
                flush()
                self._make_local(xs, keep=[q for q in range(self.n) if (x >> q) & 1])
            px, pz = self.map.mask(x), self.map.mask(z)
            batch.append((k, px & lowm, pz & lowm, pz >> self.L))
        flush()
        return self.transport.allreduce(self, vals)

    def energy(self, terms):
        return float(np.dot(self.expect(terms), [t[2] for t in terms]))

    def state(self):
        """The full state in logical qubit order (for tests; every rank gets it)."""
        parts = self.transport.gather(self, [(r, self.backend.numpy(self.slices[r])) for r in self.ranks])
        flat = [p for part in parts for p in (part if isinstance(part, list) else [part])]
        phys = np.zeros(1 << self.n, np.complex128)
        for r, a in flat:
            phys[r << self.L:(r + 1) << self.L] = a
        # physical index -> logical index
        idx = np.arange(1 << self.n, dtype=np.int64)
        logical = np.zeros_like(idx)
        for q in range(self.n):
            logical |= ((idx >> self.map.phys[q]) & 1) << q
        out = np.zeros_like(phys)
        out[logical] = phys
        return out


class GpuSlices:
    """Slices on this process's GPU: a torch complex tensor per slice, run by
    the library as an L-qubit state vector over the caller's buffer."""

    def __init__(self, dtype=None, stream=None):
        import torch

        from . import _lib as L
        self.torch = torch
        self.dtype = L.F64 if dtype is None else dtype
        self.stream = stream

    def _new(self, L_, unit):
        from .sim import State
        t = self.torch.zeros(1 << L_, dtype=self.torch.complex128 if self.dtype == 2 else self.torch.complex64,
                             device="cuda")
        st = State(1, L_, self.dtype, buf=t.data_ptr(), buf_bytes=t.numel() * t.element_size(),
                   stream=self.stream)  # initialised to |0..0>
        if not unit:
            st.sync()
            t.zero_()
        return (t, st)

    def zeros(self, L_):
        return self._new(L_, False)

    def unit(self, L_):
        return self._new(L_, True)

    def tensor(self, h):
        h[1].sync()
        return h[0]

    def apply(self, h, gates):
        self.torch.cuda.synchronize()
        h[1].apply(gates)

    def expect(self, h, terms):
        self.torch.cuda.synchronize()
        return h[1].expect(terms)

    def numpy(self, h):
        h[1].sync()
        return h[0].cpu().numpy().astype(np.complex128)
