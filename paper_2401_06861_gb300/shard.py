"""One state sharded over several GPUs by its top qubits.

The paper runs SV-Sim and DM-Sim on multi-node, multi-GPU systems for states
that do not fit one device (Sec. II; Sec. V).  Here g qubits are *global*:
they select the slice (the rank) and the other L = n - g are *local*.  A qubit
map assigns each logical qubit a physical position; positions below L are
local, position L + j is global qubit j.

A state's flat index is made of one or two *planes* of n bits, each holding
one bit per qubit at the qubit's physical position:

* state vector (one plane): amplitude index b.  Slice r holds the 2^L
  amplitudes whose top g physical bits equal r (world 2^g).
* density matrix (two planes): the library's Pauli-basis coefficients
  r[x + 2^n z] = Tr(rho P(x, z)) (x plane low, z plane high), or a row-major
  rho[r, c] (flat c + 2^n r: column plane low, row plane high).  Slice
  s = x_glob + 2^g z_glob (resp. c_glob + 2^g r_glob) holds the 4^L entries
  with those global bits, itself laid out as an L-qubit state of the same
  basis (world 4^g).

* A gate whose qubits are all local runs on every slice as a gate of an
  L-qubit state (the library's sweep kernels, unchanged).  For a density
  matrix this holds on every slice, not only on the Hermitian diagonal ones:
  a channel on local qubits acts on the flat state as (its local action) x I,
  one linear map per slice.
* A gate on a global qubit first swaps that qubit with a local one, one plane
  at a time: with global bit L + j and local bit l of a plane, rank r keeps
  the half of its slice whose local bit equals its rank bit and exchanges the
  other half with the rank that differs in that rank bit (one send and one
  receive of half a slice; contiguous when l is the plane's top local bit).
  The received half is staged in local memory and copied into place; the two
  qubits' physical positions trade places in the map.
* <P> of a Pauli string:
  - state vector: a sum over the slices of local sums, the global Z bits
    giving the sign (-1)^{|r & z_glob|}; strings with global X support first
    swap those qubits in (X support on at most L qubits; wider strings are
    refused).
  - density matrix, Pauli basis: the coefficient of P itself, held by the one
    slice whose global bits are P's (no exchange at all).
  - density matrix, row-major rho: Tr(rho P) = sum_r rho[r, r ^ x] phase(r);
    slice (c_glob, r_glob) contributes iff c_glob = r_glob ^ x_glob, its
    local trace times i^{|x_glob & z_glob|} (-1)^{|r_glob & z_glob|}.
  One all-reduce of the per-term sums ends the evaluation.

Slice storage and local arithmetic come from a backend (``GpuSlices`` /
``GpuDMSlices``: the library on the rank's GPU; the tests use the CPU oracle
on each slice), and the exchange from a transport: ``DistTransport``
(torch.distributed point to point, NCCL between GPUs or gloo on CPU, one
slice per process) or ``LocalTransport`` (all slices in one process, halves
swapped by copies).
"""
from __future__ import annotations

import numpy as np


def _popcount(v):
    return bin(v).count("1")


class QubitMap:
    """Logical qubit -> physical position (a permutation of 0..n-1)."""

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


def half_view(t, bits, l, c):
    """The 2^(bits-1) elements of a 2^bits slice whose bit l is c, as a view."""
    return t.view(1 << (bits - 1 - l), 2, 1 << l)[:, c, :]


class LocalTransport:
    """All slices in this process: a pairwise exchange swaps two halves."""

    def exchange(self, sv, j, l):
        """Swap rank bit j with local bit l of every slice."""
        for r in sv.ranks:
            p = r ^ (1 << j)
            if p < r:
                continue
            a = half_view(sv.tensor(r), sv.local_bits, l, 1 - ((r >> j) & 1))
            b = half_view(sv.tensor(p), sv.local_bits, l, 1 - ((p >> j) & 1))
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
        self.chunk = chunk  # elements per message (bounds the staging buffer)

    def exchange(self, sv, j, l):
        """Swap rank bit j with local bit l of this rank's slice."""
        (r,) = sv.ranks
        p = r ^ (1 << j)
        mine = half_view(sv.tensor(r), sv.local_bits, l, 1 - ((r >> j) & 1))
        if mine.is_contiguous():  # l is the top local bit: one contiguous half, in chunks
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


class _Sharded:
    """Qubit map, slices and the swap of a global qubit with a local one,
    common to state vectors (one plane) and density matrices (two planes)."""

    planes = 1

    def __init__(self, n, g, backend, transport, ranks, comm_device):
        if not 0 <= g < n:
            raise ValueError("need 0 <= g < n")
        self.n, self.g, self.L = n, g, n - g
        self.local_bits = self.planes * self.L
        self.world = 1 << (self.planes * g)
        self.backend, self.transport = backend, transport
        self.ranks = sorted(ranks)
        if not all(0 <= r < self.world for r in self.ranks):
            raise ValueError("rank outside the world")
        self.comm_device = comm_device
        self.map = QubitMap(n)
        self.exchanges = 0

    def tensor(self, r):
        return self.backend.tensor(self.slices[r])

    def _make_local(self, qubits, keep=()):
        """Swap every global qubit of ``qubits`` with a local one (the highest
        local position whose qubit is not in ``keep``)."""
        keep = set(keep) | set(qubits)
        for q in qubits:
            bit = self.map.phys[q]
            if bit < self.L:
                continue
            victims = [b for b in range(self.L - 1, -1, -1) if self.map.logical_at(b) not in keep]
            if not victims:
                raise ValueError("not enough local qubits for this gate or term")
            l = victims[0]
            for h in range(self.planes):  # one pairwise exchange per plane
                self.transport.exchange(self, (bit - self.L) + h * self.g, l + h * self.L)
            self.map.swap_bits(bit, l)
            self.exchanges += 1

    def _runs(self, gates):
        """Yield runs of gates (physical local qubits) between the swaps
        that make a gate's global qubits local."""
        run = []
        for name, qs, prm in gates:
            if any(self.map.phys[q] >= self.L for q in qs):
                if run:
                    yield run
                run = []
                self._make_local(qs)
            run.append((name, tuple(self.map.phys[q] for q in qs), prm))
        if run:
            yield run

    def _unpermute(self, phys):
        """A flat physical-order array of planes x n bits -> logical order."""
        idx = np.arange(phys.size, dtype=np.int64)
        logical = np.zeros_like(idx)
        for h in range(self.planes):
            for q in range(self.n):
                logical |= ((idx >> (self.map.phys[q] + h * self.n)) & 1) << (q + h * self.n)
        out = np.zeros_like(phys)
        out[logical] = phys
        return out

    def _gathered(self):
        parts = self.transport.gather(self, [(r, self.backend.numpy(self.slices[r])) for r in self.ranks])
        return [p for part in parts for p in (part if isinstance(part, list) else [part])]


class ShardedSV(_Sharded):
    """An n-qubit state vector over 2^g slices (see the module notes).

    ranks: the slice indices this process holds (all of them with
    LocalTransport, its own rank with DistTransport).  backend: slice storage
    and local arithmetic (zeros / unit / tensor / apply / expect / numpy)."""

    def __init__(self, n, g, backend, transport, ranks, comm_device="cpu"):
        super().__init__(n, g, backend, transport, ranks, comm_device)
        self.slices = {r: (backend.unit(self.L) if r == 0 else backend.zeros(self.L)) for r in self.ranks}

    def apply(self, gates):
        """Apply gates (name, logical qubits, params), grouping runs of gates
        whose qubits are local into one call per slice."""
        for run in self._runs(gates):
            for r in self.ranks:
                self.backend.apply(self.slices[r], run)

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
                    vals[k] += -vk if _popcount(r & gz) & 1 else vk
            batch.clear()

        for k, (x, z, _) in enumerate(terms):
            x, z = x & full, z & full
            xs = [q for q in range(self.n) if (x >> q) & 1 and self.map.phys[q] >= self.L]
            if xs:
                if _popcount(x) > self.L:
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
        phys = np.zeros(1 << self.n, np.complex128)
        for r, a in self._gathered():
            phys[r << self.L:(r + 1) << self.L] = a
        return self._unpermute(phys)


class ShardedDM(_Sharded):
    """An n-qubit density matrix over 4^g slices (see the module notes).

    backend.basis is "pauli" (slices of the library's Pauli-basis
    coefficients) or "matrix" (slices of a row-major rho).  backend: zeros /
    unit / tensor / apply(slice, gates, noise) / expect(slice, terms) ->
    complex local traces Tr(P_loc X) / numpy.  ``noise`` (as the library's
    noise model, T1 / T2 per logical qubit) applies after every gate."""

    planes = 2

    def __init__(self, n, g, backend, transport, ranks, comm_device="cpu"):
        super().__init__(n, g, backend, transport, ranks, comm_device)
        if backend.basis not in ("pauli", "matrix"):
            raise ValueError("unknown slice basis")
        self.basis = backend.basis
        gm = (1 << g) - 1
        # |0..0><0..0|: Pauli basis r[x, z] = [x = 0] (every z); rho: one entry.
        unit = (lambda r: (r & gm) == 0) if self.basis == "pauli" else (lambda r: r == 0)
        self.slices = {r: (backend.unit(self.L) if unit(r) else backend.zeros(self.L)) for r in self.ranks}

    def _local_noise(self, noise):
        """The noise model with T1 / T2 at the local physical positions."""
        if noise is None:
            return None
        out = dict(noise)
        lq = [self.map.logical_at(b) for b in range(self.L)]
        out["T1_us"] = np.asarray(noise["T1_us"], np.float64)[lq]
        out["T2_us"] = np.asarray(noise["T2_us"], np.float64)[lq]
        return out

    def apply(self, gates, noise=None):
        """Apply gates (name, logical qubits, params), each followed by its
        noise, grouping runs of gates whose qubits are local into one call
        per slice."""
        for run in self._runs(gates):
            nl = self._local_noise(noise)
            for r in self.ranks:
                self.backend.apply(self.slices[r], run, nl)

    def _factor(self, r, xg, zg):
        """Weight of slice r's local trace in Tr(rho P) (module notes)."""
        lo, hi = r & ((1 << self.g) - 1), r >> self.g
        if self.basis == "pauli":
            return 1.0 if (lo, hi) == (xg, zg) else 0.0
        if lo != hi ^ xg:  # column bits = row bits ^ x on the global qubits
            return 0.0
        return (1j ** (_popcount(xg & zg) & 3)) * (-1.0 if _popcount(hi & zg) & 1 else 1.0)

    def expect(self, terms):
        """Per-term Tr(rho P) (coefficients not applied); no exchange."""
        vals = np.zeros(len(terms))
        full = (1 << self.n) - 1
        lowm = (1 << self.L) - 1
        mapped = [(self.map.mask(x & full), self.map.mask(z & full)) for x, z, _ in terms]
        for r in self.ranks:
            mine = []
            for k, (px, pz) in enumerate(mapped):
                f = self._factor(r, px >> self.L, pz >> self.L)
                if f != 0:
                    mine.append((k, px & lowm, pz & lowm, f))
            if not mine:
                continue
            v = self.backend.expect(self.slices[r], [(lx, lz, 1.0) for _, lx, lz, _ in mine])
            for (k, _, _, f), vk in zip(mine, v):
                vals[k] += (f * vk).real
        return self.transport.allreduce(self, vals)

    def energy(self, terms):
        return float(np.dot(self.expect(terms), [t[2] for t in terms]))

    def state(self):
        """The full flat state (4^n entries, the backend's basis) in logical
        qubit order (for tests; every rank gets it)."""
        n, L, g = self.n, self.L, self.g
        parts = self._gathered()
        phys = np.zeros(1 << (2 * n), np.result_type(*[a.dtype for _, a in parts]))
        s = np.arange(1 << (2 * L), dtype=np.int64)
        base = (s & ((1 << L) - 1)) | ((s >> L) << n)  # slice bits of both planes
        for r, a in parts:
            lo, hi = r & ((1 << g) - 1), r >> g
            phys[base | (lo << L) | (hi << (n + L))] = a
        return self._unpermute(phys)


class GpuSlices:
    """State-vector slices on this process's GPU: a torch complex tensor per
    slice, run by the library as an L-qubit state vector over the caller's
    buffer."""

    def __init__(self, dtype=None, stream=None):
        import torch

        from . import _lib as L
        self.torch = torch
        self.dtype = L.F64 if dtype is None else dtype
        self.stream = stream

    def _new(self, L_, unit):
        from . import _lib as L
        from .sim import State
        t = self.torch.zeros(1 << L_, dtype=self.torch.complex128 if self.dtype == L.F64 else self.torch.complex64,
                             device="cuda")
        st = State(L.SV, L_, self.dtype, buf=t.data_ptr(), buf_bytes=t.numel() * t.element_size(),
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


class GpuDMSlices:
    """Density-matrix slices on this process's GPU: a torch real tensor of
    4^L Pauli-basis coefficients per slice, run by the library as an L-qubit
    density matrix over the caller's buffer."""

    basis = "pauli"

    def __init__(self, dtype=None, stream=None):
        import torch

        from . import _lib as L
        self.torch = torch
        self.dtype = L.F64 if dtype is None else dtype
        self.stream = stream

    def _new(self, L_, unit):
        from . import _lib as L
        from .sim import State
        t = self.torch.zeros(1 << (2 * L_), dtype=self.torch.float64 if self.dtype == L.F64 else self.torch.float32,
                             device="cuda")
        st = State(L.DM, L_, self.dtype, buf=t.data_ptr(), buf_bytes=t.numel() * t.element_size(),
                   stream=self.stream)  # initialised to |0..0><0..0|
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

    def apply(self, h, gates, noise):
        self.torch.cuda.synchronize()
        h[1].apply(gates, noise)

    def expect(self, h, terms):
        self.torch.cuda.synchronize()
        return h[1].expect(terms).astype(np.complex128)

    def numpy(self, h):
        h[1].sync()
        return h[0].cpu().numpy().astype(np.float64)
