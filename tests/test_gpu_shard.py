"""High-qubit sharding with the library's kernels on every slice, on one GPU:
all 2^g slices live in this process (LocalTransport: the pairwise half-slice
exchanges are copies between the slices' buffers), so the sharded path runs
the same sweep and expectation kernels a multi-GPU run would, against the
unsharded oracle at 1e-12 (FP64) and 1e-5 (FP32)."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.shard import GpuSlices, LocalTransport, ShardedSV

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
