"""The tensor-core kernel's bounded waits, made to run out on purpose: the
wait-test hook withholds the MMAs, so the MMA-completion barrier is one that
nothing arrives on.  Every CTA's wait must run out, be counted and reported
as NWQ_ETIMEOUT, leave the state unwritten and the context usable: a normal
run of the same plan on the same state then passes parity."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim
from paper_2401_06861_gb300.sim import Plan, State

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


@pytest.mark.parametrize("n", [12, 15])
def test_withheld_mmas_time_out_and_the_context_stays_usable(n):
    gates = inputs.random_circuit(n, 40, 900 + n)
    psi0 = inputs.random_state(n, 901 + n).astype(np.complex64)
    with State(L.SV, n, L.F32) as st, Plan(L.SV, n, gates, L.F32, flags=L.PLAN_TC) as p:
        st.load(psi0)
        before = sim.tc_timeouts()
        count = ctypes.c_int(-1)
        rc = L.lib().nwq_tc_wait_test(st.h, p.h, ctypes.byref(count))
        assert rc == L.ETIMEOUT and b"ran out" in L.lib().nwq_last_error()
        ctas = min(1 << (n - 12), 3 * 152)
        assert count.value == ctas and sim.tc_timeouts() == before + count.value  # one per CTA
        assert np.array_equal(st.copy(), psi0)  # the tiles were left unwritten
        st.run(p)  # the same plan, MMAs issued: completes and matches the oracle
        got = st.copy()
        assert sim.tc_timeouts() == before + count.value
    ref = oracle.sv_run(n, gates, psi0.astype(np.complex128))
    assert float(np.max(np.abs(got - ref))) <= 1e-5
