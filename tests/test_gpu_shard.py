"""High-qubit sharding with the library's kernels on every slice, on one GPU:
all slices live in this process (LocalTransport: the pairwise half-slice
exchanges are copies between the slices' buffers), so the sharded path runs
the same sweep and expectation kernels a multi-GPU run would, against the
unsharded oracle at 1e-12 (FP64) and 1e-5 (FP32).  Density matrices are
sharded as slices of the library's Pauli-basis coefficients."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.shard import GpuDMSlices, GpuSlices, LocalTransport, ShardedDM, ShardedSV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


@pytest.mark.parametrize("n,g,dtype", [(14, 1, L.F64), (16, 2, L.F64), (20, 3, L.F64), (18, 2, L.F32)])
def test_sharded_state_vector_on_one_gpu_matches_the_oracle(n, g, dtype):
    gates = inputs.random_circuit(n, 120, 700 + n) + inputs.large_sv_tfim(n, 2)[0]
    terms = inputs.tfim_terms(n) + inputs.z_terms(n) + inputs.random_pauli_terms(n, 20, 701 + n)
    sv = ShardedSV(n, g, GpuSlices(dtype), LocalTransport(), ranks=range(1 << g))
    sv.apply(gates)
    got = sv.expect(terms)
    psi = sv.state()
    ref = oracle.sv_run(n, gates)
    tol = 1e-12 if dtype == L.F64 else 1e-5
    assert sv.exchanges > 0
    assert np.max(np.abs(psi - ref)) <= tol
    assert np.max(np.abs(got - oracle.sv_expect(ref, n, terms))) <= (1e-12 if dtype == L.F64 else 2e-5)


def all_strings(n):
    return [(k & ((1 << n) - 1), k >> n, 1.0) for k in range(1 << (2 * n))]


@pytest.mark.parametrize("n,g,dtype", [(7, 1, L.F64), (8, 2, L.F64), (7, 1, L.F32)])
def test_sharded_density_matrix_on_one_gpu_matches_the_oracle(n, g, dtype):
    gates = inputs.random_circuit(n, 60, 900 + n) + inputs.tfim_trotter(n, 1.0, 0.7, 0.05, 1)
    noise = inputs.noise_params(n, seed=901 + n)
    terms = inputs.tfim_terms(n) + inputs.z_terms(n) + inputs.random_pauli_terms(n, 20, 902 + n)
    terms += [((1 << n) - 1, (1 << n) - 1, 1.0), (1 << (n - 1), 0, 1.0)]  # X / Y on global qubits
    dm = ShardedDM(n, g, GpuDMSlices(dtype), LocalTransport(), ranks=range(4 ** g))
    dm.apply(gates, noise)
    got = dm.expect(terms)
    coefs = dm.state()
    ref = oracle.dm_run(n, gates, noise)
    tol = 1e-12 if dtype == L.F64 else 1e-5
    assert dm.exchanges > 0
    assert np.max(np.abs(coefs - oracle.dm_expect(ref, n, all_strings(n)))) <= tol
    assert np.max(np.abs(got - oracle.dm_expect(ref, n, terms))) <= tol
