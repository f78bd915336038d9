"""High-qubit sharding of one state vector or density matrix (paper Sec. II /
V: SV-Sim and DM-Sim across nodes and GPUs), on the CPU: every slice is an
oracle state of n - g qubits (for density matrices: a block of a row-major
rho, or a slice of the Pauli-basis coefficients), the exchanges run in
process (LocalTransport) or between `gloo` ranks (DistTransport, one process
per slice), and the gathered state and the Pauli expectations are compared
with the unsharded oracle at 1e-12."""
import os
import socket
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.shard import DistTransport, LocalTransport, QubitMap, ShardedDM, ShardedSV, half_view
from tests.dense import pauli_dense

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleSlices:
    """Each slice a CPU complex128 tensor, gates and sums by the oracle."""

    @staticmethod
    def _n(t):
        return t.numel().bit_length() - 1

    def zeros(self, L):
        return torch.zeros(1 << L, dtype=torch.complex128)

    def unit(self, L):
        t = self.zeros(L)
        t[0] = 1.0
        return t

    def tensor(self, h):
        return h

    def apply(self, h, gates):
        oracle.sv_run_inplace(h.numpy(), self._n(h), gates)

    def expect(self, h, terms):
        return oracle.sv_expect(h.numpy(), self._n(h), terms)

    def numpy(self, h):
        return h.numpy().copy()


def workload(n, seed):
    gates = inputs.random_circuit(n, 90, seed) + inputs.tfim_trotter(n, 1.0, 0.7, 0.05, 2)
    terms = inputs.random_pauli_terms(n, 25, seed + 1) + inputs.tfim_terms(n) + inputs.z_terms(n)
    wide = ((1 << n) - 1) >> 3  # X on the n - 3 lowest qubits (fits any slice here)
    top = ((1 << n) - 1) ^ ((1 << (n - 3)) - 1)  # the three top qubits, which start global
    mixed = top | ((1 << (n - 6)) - 1)  # X on n - 3 qubits, three of them global, Y on all
    terms += [(wide, 0, 1.0), (mixed, (1 << n) - 1, -0.5), (1 << (n - 1), 1 << (n - 2), 0.25)]
    return gates, terms


def test_wider_x_support_than_a_slice_is_refused():
    n, g = 6, 2
    sv = ShardedSV(n, g, OracleSlices(), LocalTransport(), ranks=range(1 << g))
    with pytest.raises(ValueError, match="more than n - g"):
        sv.expect([((1 << n) - 1, 0, 1.0)])


def test_qubit_map_and_half_views():
    m = QubitMap(5)
    m.swap_bits(4, 1)
    assert m.phys == [0, 4, 2, 3, 1] and m.logical_at(4) == 1 and m.mask(0b00010) == 0b10000
    t = torch.arange(16)
    assert half_view(t, 4, 3, 1).reshape(-1).tolist() == list(range(8, 16))  # top bit: contiguous half
    assert half_view(t, 4, 0, 1).reshape(-1).tolist() == [1, 3, 5, 7, 9, 11, 13, 15]


@pytest.mark.parametrize("n,g", [(6, 1), (8, 2), (9, 3), (12, 2)])
def test_sharded_state_and_expectations_match_the_oracle(n, g):
    gates, terms = workload(n, 100 + n + g)
    sv = ShardedSV(n, g, OracleSlices(), LocalTransport(), ranks=range(1 << g))
    sv.apply(gates)
    ref = oracle.sv_run(n, gates)
    assert sv.exchanges > 0  # the circuit touches global qubits
    assert np.max(np.abs(sv.state() - ref)) <= 1e-12
    got = sv.expect(terms)
    assert np.max(np.abs(got - oracle.sv_expect(ref, n, terms))) <= 1e-12
    assert abs(sv.energy(terms) - oracle.energy(oracle.sv_expect(ref, n, terms), terms)) <= 1e-12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    g = ws.bit_length() - 1
    gates, terms = workload(n, 300 + n)
    sv = ShardedSV(n, g, OracleSlices(), DistTransport(chunk=1 << (n - g - 2)), ranks=[rank])
    sv.apply(gates)
    vals = sv.expect(terms)
    state = sv.state()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, sv.exchanges, vals, state))


@pytest.mark.parametrize("ws,n", [(2, 9), (4, 10)])
def test_gloo_ranks_each_holding_one_slice(ws, n):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, n, qu)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted((qu.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gates, terms = workload(n, 300 + n)
    ref = oracle.sv_run(n, gates)
    eref = oracle.sv_expect(ref, n, terms)
    for rank, exchanges, vals, state in out:
        assert exchanges == out[0][1] > 0          # every rank took the same exchanges
        assert np.max(np.abs(vals - eref)) <= 1e-12  # one all-reduce: the same values on every rank
        assert np.max(np.abs(state - ref)) <= 1e-12


# ---------------------------------------------------------------- density matrices
class OracleDMSlices:
    """Each slice a block of a row-major rho (flat c + 2^L r), as a CPU
    complex128 tensor; channels and traces by the oracle.  A block off the
    diagonal is not Hermitian, so its local trace Tr(P X) is taken as
    Re Tr(P X) + i Re Tr(P (-i X))."""

    basis = "matrix"

    @staticmethod
    def _L(t):
        return (t.numel().bit_length() - 1) // 2

    def zeros(self, L):
        return torch.zeros(1 << (2 * L), dtype=torch.complex128)

    def unit(self, L):
        t = self.zeros(L)
        t[0] = 1.0
        return t

    def tensor(self, h):
        return h

    def apply(self, h, gates, noise):
        L = self._L(h)
        out = oracle.dm_run(L, gates, noise, rho0=h.numpy().reshape(1 << L, 1 << L))
        h.copy_(torch.from_numpy(out.reshape(-1)))

    def expect(self, h, terms):
        L = self._L(h)
        X = h.numpy().reshape(1 << L, 1 << L)
        return oracle.dm_expect(X, L, terms) + 1j * oracle.dm_expect(-1j * X, L, terms)

    def numpy(self, h):
        return h.numpy().copy()


class OraclePauliSlices:
    """Each slice 4^L real Pauli-basis coefficients r[x + 2^L z] (the
    library's layout), as a CPU float64 tensor.  A slice is the Hermitian
    operator X = 2^-L sum r[x, z] P(x, z); a channel is applied to X by the
    oracle and the coefficients read back as Tr(X P(x, z))."""

    basis = "pauli"
    _paulis = {}

    @staticmethod
    def _L(t):
        return (t.numel().bit_length() - 1) // 2

    def _all(self, L):
        if L not in self._paulis:
            self._paulis[L] = [pauli_dense(L, k & ((1 << L) - 1), k >> L) for k in range(1 << (2 * L))]
        return self._paulis[L]

    def _op(self, h):
        L = self._L(h)
        r = h.numpy()
        return sum(r[k] * P for k, P in enumerate(self._all(L))) / (1 << L)

    def _coefs(self, X, L):
        return oracle.dm_expect(X, L, all_strings(L))

    def zeros(self, L):
        return torch.zeros(1 << (2 * L), dtype=torch.float64)

    def unit(self, L):
        t = self.zeros(L)
        t.view(1 << L, 1 << L)[:, 0] = 1.0  # x = 0, every z
        return t

    def tensor(self, h):
        return h

    def apply(self, h, gates, noise):
        L = self._L(h)
        out = oracle.dm_run(L, gates, noise, rho0=self._op(h))
        h.copy_(torch.from_numpy(self._coefs(out, L)))

    def expect(self, h, terms):
        return oracle.dm_expect(self._op(h), self._L(h), terms).astype(np.complex128)

    def numpy(self, h):
        return h.numpy().copy()


def all_strings(n):
    """Every Pauli string (x, z) in the order of the flat index x + 2^n z."""
    return [(k & ((1 << n) - 1), k >> n, 1.0) for k in range(1 << (2 * n))]


def dm_workload(n, seed):
    gates = inputs.random_circuit(n, 40, seed) + inputs.tfim_trotter(n, 1.0, 0.7, 0.05, 1)
    noise = inputs.noise_params(n, seed=seed + 2)
    terms = inputs.random_pauli_terms(n, 25, seed + 1) + inputs.tfim_terms(n) + inputs.z_terms(n)
    full = (1 << n) - 1
    terms += [(full, 0, 1.0), (full, full, -0.5), (1 << (n - 1), 1 << (n - 2), 0.25), (0, 0, 1.0)]
    return gates, noise, terms


def test_dm_slices_start_as_the_ground_state_in_both_bases():
    n, g = 4, 1
    for be, ref in ((OracleDMSlices(), oracle.dm_zero(n).reshape(-1)),
                    (OraclePauliSlices(), oracle.dm_expect(oracle.dm_zero(n), n, all_strings(n)))):
        dm = ShardedDM(n, g, be, LocalTransport(), ranks=range(4 ** g))
        assert np.array_equal(dm.state(), ref)


@pytest.mark.parametrize("n,g", [(4, 1), (5, 1), (6, 2)])
def test_sharded_density_matrix_matches_the_oracle(n, g):
    gates, noise, terms = dm_workload(n, 500 + n + g)
    dm = ShardedDM(n, g, OracleDMSlices(), LocalTransport(), ranks=range(4 ** g))
    dm.apply(gates, noise)
    ref = oracle.dm_run(n, gates, noise)
    assert dm.exchanges > 0
    assert np.max(np.abs(dm.state() - ref.reshape(-1))) <= 1e-12
    eref = oracle.dm_expect(ref, n, terms)
    assert np.max(np.abs(dm.expect(terms) - eref)) <= 1e-12
    assert abs(dm.energy(terms) - oracle.energy(eref, terms)) <= 1e-12


@pytest.mark.parametrize("n,g", [(4, 1), (5, 1), (5, 2)])
def test_sharded_pauli_coefficients_match_the_oracle(n, g):
    gates, noise, terms = dm_workload(n, 600 + n + g)
    dm = ShardedDM(n, g, OraclePauliSlices(), LocalTransport(), ranks=range(4 ** g))
    dm.apply(gates, noise)
    ref = oracle.dm_run(n, gates, noise)
    assert dm.exchanges > 0
    assert np.max(np.abs(dm.state() - oracle.dm_expect(ref, n, all_strings(n)))) <= 1e-12
    assert np.max(np.abs(dm.expect(terms) - oracle.dm_expect(ref, n, terms))) <= 1e-12


def _dm_rank(rank, ws, port, n, q, basis="matrix"):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    g = (ws.bit_length() - 1) // 2
    gates, noise, terms = dm_workload(n, 800 + n)
    backend = OracleDMSlices() if basis == "matrix" else OraclePauliSlices()
    dm = ShardedDM(n, g, backend, DistTransport(chunk=1 << (2 * (n - g) - 3)), ranks=[rank])
    dm.apply(gates, noise)
    vals = dm.expect(terms)
    state = dm.state()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, dm.exchanges, vals, state))


@pytest.mark.parametrize("basis", ["matrix", "pauli"])
def test_gloo_ranks_each_holding_one_density_matrix_slice(basis):
    import torch.multiprocessing as mp
    ws, n = 4, 5
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dm_rank, args=(r, ws, port, n, qu, basis)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted((qu.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gates, noise, terms = dm_workload(n, 800 + n)
    ref = oracle.dm_run(n, gates, noise)
    eref = oracle.dm_expect(ref, n, terms)
    sref = ref.reshape(-1) if basis == "matrix" else oracle.dm_expect(ref, n, all_strings(n))
    for rank, exchanges, vals, state in out:
        assert exchanges == out[0][1] > 0
        assert np.max(np.abs(vals - eref)) <= 1e-12
        assert np.max(np.abs(state - sref)) <= 1e-12
