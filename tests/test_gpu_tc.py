"""GPU parity of tensor-core plans (NWQ_PLAN_TC: the circuit fused into dense
five-qubit blocks, each applied by tcgen05 MMAs of kind TF32 with the
three-term hi/lo split) against the FP64 CPU oracle, through the C ABI.

Tolerances are those of the FP32 path: 1e-5 max absolute amplitude error and
1e-6 relative energy error |E - E_ref| / max(|E_ref|, sum |coeff|)."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim
from paper_2401_06861_gb300.sim import Plan, State

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    torch.cuda.init()
    before = sim.tc_timeouts()
    yield
    assert sim.tc_timeouts() == before  # no bounded wait ran out in this module


def maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


def rel_energy(e, eref, terms):
    return abs(e - eref) / max(abs(eref), sum(abs(t[2]) for t in terms))


def run(n, gates, psi0, flags):
    with State(L.SV, n, L.F32) as st, Plan(L.SV, n, gates, L.F32, flags=flags) as p:
        st.load(psi0.astype(np.complex64))
        st.run(p)
        return st.copy(), p.info()["sweeps"]


# n = 12: one tile; n = 22: 1024 tiles over at most 2 CTAs per SM, so every
# CTA walks several tiles with the next tile's loads in flight
@pytest.mark.parametrize("n", [12, 13, 14, 16, 22])
def test_tc_random_circuits(n):
    gates = inputs.random_circuit(n, 100 if n < 20 else 40, 5000 + n)
    psi0 = inputs.random_state(n, 5100 + n)
    got, nb = run(n, gates, psi0, L.PLAN_TC)
    ref = oracle.sv_run(n, gates, psi0)
    err = maxerr(got, ref)
    print(f"tc n={n}: {len(gates)} gates in {nb} blocks, max abs err {err:.3e}")
    assert err <= TOL


@pytest.mark.parametrize("qs", [(0, 1, 2, 3, 4), (3, 4, 5, 6, 7), (7, 8, 9, 10, 11), (0, 5, 9, 13, 17),
                                (13, 14, 15, 16, 17), (1, 2, 3, 4, 17), (2, 6, 7, 8, 16)])
def test_tc_single_block_geometries(qs):
    # one dense block on the given qubits: qubit 0 in or out of the block,
    # block bits low, interleaved with the row bits, or far above them
    n = 18
    rng = np.random.default_rng(sum(qs))
    gates = []
    for _ in range(2):
        for a, b in zip(qs[:-1], qs[1:]):
            gates.append(("MAT2", (a, b), inputs.random_unitary(4, rng)))
        for q in qs:
            gates.append(("MAT1", (q,), inputs.random_unitary(2, rng)))
    with Plan(L.SV, n, gates, L.F32, flags=L.PLAN_TC) as p:
        blocks = p.tc_blocks()
    assert len(blocks) == 1 and blocks[0][0] == tuple(qs)
    psi0 = inputs.random_state(n, 77)
    got, _ = run(n, gates, psi0, L.PLAN_TC)
    fused, _ = run(n, gates, psi0, L.PLAN_FUSED)
    ref = oracle.sv_run(n, gates, psi0)
    print(f"block {qs}: tc err {maxerr(got, ref):.3e}, fused err {maxerr(fused, ref):.3e}")
    assert maxerr(got, ref) <= TOL
    assert maxerr(got, fused) <= TOL


def test_tc_tfim_n20_depth10_energy():
    n = 20
    gates, h = inputs.large_sv_tfim(n, 10)
    terms = inputs.tfim_terms(n, 1.0, h)
    ref = oracle.sv_run(n, gates)
    eref = oracle.energy(oracle.sv_expect(ref, n, terms), terms)
    with State(L.SV, n, L.F32) as st, Plan(L.SV, n, gates, L.F32, flags=L.PLAN_TC) as p:
        st.run(p)
        got = st.copy()
        e = st.expect(terms, sum=True, normalize=True)
        z = np.real(st.expect(inputs.z_terms(n), normalize=True))
        nrm = st.norm()
    zref = np.real(oracle.sv_expect(ref, n, inputs.z_terms(n)))
    print(f"tc tfim n=20: amp err {maxerr(got, ref):.3e}, rel E {rel_energy(e, eref, terms):.3e}, "
          f"<Z> err {maxerr(z, zref):.3e}, norm-1 {nrm - 1:.2e}")
    assert maxerr(got, ref) <= TOL
    assert maxerr(z, zref) <= TOL
    assert rel_energy(e, eref, terms) <= 1e-6


def test_tc_n30_tfim_matches_free_fermions():
    # 8 GiB state, 2^18 tiles: the benchmark's circuit family against exact values
    from oracle import tfim_fermion
    n = 30
    gates, h = inputs.large_sv_tfim(n, 10)
    ref = tfim_fermion.tfim_observables(n, gates)
    terms = inputs.tfim_terms(n, 1.0, h)
    eref = -float(np.sum(ref["zz"])) - float(np.dot(h, ref["x"]))
    with Plan(L.SV, n, gates, L.F32, flags=L.PLAN_TC) as p, State(L.SV, n, L.F32) as st:
        st.run(p)
        zz = np.real(st.expect(inputs.zz_terms(n), normalize=True))
        x = np.real(st.expect(inputs.x_terms(n), normalize=True))
        e = st.expect(terms, sum=True, normalize=True)
    err = max(maxerr(zz, ref["zz"]), maxerr(x, ref["x"]))
    print(f"tc n=30: max term error {err:.3e}, rel E {rel_energy(e, eref, terms):.3e}")
    assert err <= TOL
    assert rel_energy(e, eref, terms) <= 1e-6


def test_tc_empty_plan_leaves_state():
    n = 12
    psi0 = inputs.random_state(n, 3)
    got, nb = run(n, [], psi0, L.PLAN_TC)
    assert nb == 0 and maxerr(got, psi0.astype(np.complex64)) == 0.0
