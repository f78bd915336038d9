"""nwq_expect_pauli_sum_noalloc (the allocation-free expectation entry point)
against nwq_expect_pauli_sum, both called through the C ABI.

The no-allocation variant serves callers that cannot allocate device memory
(another allocator owns it all, or a latency-critical loop must not wait for
or fail on an allocation).  It keeps its scratch in one library-owned device
array shared by all calls, so the check runs it twice in a row on different
inputs: the second call must not see leftovers of the first.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.sim import State

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


def call(fn, st, terms, flags):
    arr = L.encode_terms(terms)
    n_out = 1 if flags & L.EXPECT_SUM else len(terms)
    out = np.full(max(n_out, 1), np.nan)
    rc = fn(st.h, arr, len(terms), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), flags)
    return rc, out[:n_out]


@pytest.mark.parametrize("kind,n,dtype,tol", [(L.SV, 14, L.F64, 1e-12), (L.SV, 9, L.F32, 1e-12),
                                              (L.DM, 6, L.F64, 1e-12)])
def test_noalloc_matches_allocating_entry_point_twice(kind, n, dtype, tol):
    lib = L.lib()
    with State(kind, n, dtype) as st:
        for call_no, seed in enumerate((11, 12)):
            if kind == L.SV:
                st.load(inputs.random_state(n, seed))
            else:
                st.load(inputs.random_density(n, seed))
            # different term counts per call, more than one term chunk per x mask
            terms = inputs.random_pauli_terms(n, 40 + 30 * call_no, seed) + inputs.tfim_terms(n) + inputs.z_terms(n)
            for flags in (L.EXPECT_TERMS, L.EXPECT_SUM, L.EXPECT_TERMS | L.EXPECT_NORMALIZE,
                          L.EXPECT_SUM | L.EXPECT_NORMALIZE):
                rc_a, ref = call(lib.nwq_expect_pauli_sum, st, terms, flags)
                rc_b, got = call(lib.nwq_expect_pauli_sum_noalloc, st, terms, flags)
                assert rc_a == L.OK and rc_b == L.OK, lib.nwq_last_error()
                assert np.all(np.isfinite(got))
                err = float(np.max(np.abs(got - ref)))
                assert err <= tol, (call_no, flags, err)


def test_noalloc_rejects_too_many_terms():
    lib = L.lib()
    with State(L.SV, 4, L.F64) as st:
        terms = inputs.random_pauli_terms(4, L.NOALLOC_MAX_TERMS + 1, 3)
        rc, _ = call(lib.nwq_expect_pauli_sum_noalloc, st, terms, L.EXPECT_TERMS)
        assert rc == L.EINVAL
        assert b"NWQ_NOALLOC_MAX_TERMS" in lib.nwq_last_error()
        rc, out = call(lib.nwq_expect_pauli_sum_noalloc, st, terms[:L.NOALLOC_MAX_TERMS], L.EXPECT_SUM)
        assert rc == L.OK and np.isfinite(out[0])
