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


def launch_shape(st, nt, noalloc):
    g, fb = ctypes.c_int(0), ctypes.c_int(0)
    assert L.lib().nwq_expect_launch_shape(st.h, nt, noalloc, ctypes.byref(g), ctypes.byref(fb)) == L.OK
    return g.value, fb.value


def wide_terms(n, count, seed):
    """Strings over every tile pass and the general kernel: Z-type and
    low-X strings, X supports on high bits, and X supports wider than any
    tile (more than 8 bits above bit 3)."""
    rng = np.random.default_rng(seed)
    t = inputs.tfim_terms(n) + inputs.z_terms(n)
    for k in range(count - len(t)):
        w = (2, 6, 11, 16)[k % 4]
        bits = rng.choice(n, size=w, replace=False)
        x = int(sum(1 << int(b) for b in bits))
        t.append((x, int(rng.integers(0, 1 << n)), float(rng.uniform(-1, 1))))
    return t


@pytest.mark.parametrize("dtype", [L.F32, L.F64])
def test_noalloc_reduced_launch_shape_matches_twice(dtype):
    # 256 terms on 2^22 amplitudes: the allocation-free call caps the general
    # kernel's blocks at 256 and shrinks the tiled grid until its partial sums
    # fit the static array; only the FP64 summation order may change
    lib = L.lib()
    n, nt = 22, L.NOALLOC_MAX_TERMS
    with State(L.SV, n, dtype) as st:
        g_a, fb_a = launch_shape(st, nt, 0)
        g_n, fb_n = launch_shape(st, nt, 1)
        assert g_n < g_a and fb_n == 256 < fb_a, (g_a, fb_a, g_n, fb_n)
        for call_no, seed in enumerate((21, 22)):
            st.load(inputs.random_state(n, seed))
            terms = wide_terms(n, nt - call_no, seed)
            for flags in (L.EXPECT_TERMS, L.EXPECT_SUM | L.EXPECT_NORMALIZE):
                rc_a, ref = call(lib.nwq_expect_pauli_sum, st, terms, flags)
                rc_b, got = call(lib.nwq_expect_pauli_sum_noalloc, st, terms, flags)
                assert rc_a == L.OK and rc_b == L.OK, lib.nwq_last_error()
                err = float(np.max(np.abs(got - ref)))
                assert err <= 1e-12, (call_no, flags, err)


class DefaultPool:
    """Used-memory figures of the device's default stream-ordered memory pool
    (driver API through ctypes); the allocating entry point takes its scratch
    from that pool."""
    USED_CURRENT, USED_HIGH = 7, 8  # CUmemPool_attribute

    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = ctypes.c_int(0)
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):  # the high watermark restarts from the current use
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(v)) == 0


def test_noalloc_allocates_no_device_memory():
    import torch
    lib = L.lib()
    n = 22
    pool = DefaultPool(torch.cuda.current_device())
    with State(L.SV, n, L.F32) as st:
        st.load(inputs.random_state(n, 31))
        terms = wide_terms(n, L.NOALLOC_MAX_TERMS, 31)
        for fn in (lib.nwq_expect_pauli_sum_noalloc, lib.nwq_expect_pauli_sum):  # load every kernel once
            assert call(fn, st, terms, L.EXPECT_TERMS)[0] == L.OK
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pool.reset_high()
        used0 = pool.get(pool.USED_CURRENT)
        for flags in (L.EXPECT_TERMS, L.EXPECT_SUM):
            assert call(lib.nwq_expect_pauli_sum_noalloc, st, terms, flags)[0] == L.OK
        assert pool.get(pool.USED_HIGH) == used0 == pool.get(pool.USED_CURRENT)
        assert torch.cuda.mem_get_info()[0] == free0
        # the same probe sees the allocating entry point's scratch
        pool.reset_high()
        assert call(lib.nwq_expect_pauli_sum, st, terms, L.EXPECT_TERMS)[0] == L.OK
        assert pool.get(pool.USED_HIGH) > used0
