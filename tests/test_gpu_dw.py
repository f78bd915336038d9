"""Double-word sweeps (the default of FP64 plans): specialised kernels that hold
every value as two floats and run on the FP32 pipe, against the FP64 oracle
at the FP64 tolerance (1e-12).

A double-word run and an FP64-pipe run of the same plan round differently, so
their results agree to the tolerance but not bit for bit: each test also
checks that the two differ somewhere, which shows the double-word kernels ran.
"""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.sim import Plan, State

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


def maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def run_both(kind, n, gates, noise=None, psi0=None, flags=0):
    out = {}
    for extra in (L.PLAN_FP64, L.PLAN_DW):
        with State(kind, n, L.F64) as st, Plan(kind, n, gates, L.F64, noise, flags=flags | extra) as p:
            if psi0 is not None:
                st.load(psi0)
            st.run(p)
            assert p.last_run_dw() == (extra == L.PLAN_DW)
            out[extra] = st.copy()
    return out[L.PLAN_FP64], out[L.PLAN_DW]


@pytest.mark.parametrize("n,family", [(18, "random"), (19, "random_mat"), (20, "tfim"), (18, "hea"), (21, "plain")])
def test_dw_state_vectors_match_the_oracle(n, family):
    flags = 0
    if family == "random":
        gates = inputs.random_circuit(n, 300, 5000 + n, names=[g for g in inputs.GATE_NAMES if not g.startswith("MAT")])
    elif family == "random_mat":
        gates = inputs.random_circuit(n, 150, 5100 + n)
    elif family == "tfim":
        gates = inputs.large_sv_tfim(n, 6)[0]
    elif family == "hea":
        gates = inputs.hea_ansatz(n, 4, inputs.hea_params(n, 4, 1)[0])[0]
    else:
        gates, flags = inputs.random_circuit(n, 60, 5200 + n), L.PLAN_PLAIN
    psi0 = inputs.random_state(n, 5300 + n)
    f64, dw = run_both(L.SV, n, gates, psi0=psi0, flags=flags)
    ref = oracle.sv_run(n, gates, psi0)
    err, err64 = maxerr(dw, ref), maxerr(f64, ref)
    print(f"dw sv n={n} {family}: double-word err {err:.3e}, FP64 err {err64:.3e}")
    assert err <= 1e-12
    assert not np.array_equal(dw, f64)


@pytest.mark.parametrize("n,seed", [(9, 1), (10, 2)])
def test_dw_noisy_density_matrices_match_the_oracle(n, seed):
    gates = inputs.random_circuit(n, 80, 5400 + seed)
    noise = inputs.noise_params(n, seed=5500 + seed)
    rho0 = inputs.random_density(n, 5600 + seed)
    out = {}
    for extra in (L.PLAN_FP64, L.PLAN_DW):
        with State(L.DM, n, L.F64) as st, Plan(L.DM, n, gates, L.F64, noise, flags=extra) as p:
            st.load(rho0)
            st.run(p)
            assert p.last_run_dw() == (extra == L.PLAN_DW)
            out[extra] = st.copy()
    ref = oracle.dm_run(n, gates, noise, rho0)
    err = maxerr(out[L.PLAN_DW], ref)
    print(f"dw dm n={n}: double-word err {err:.3e}, FP64 err {maxerr(out[L.PLAN_FP64], ref):.3e}")
    assert err <= 1e-12
    assert not np.array_equal(out[L.PLAN_FP64], out[L.PLAN_DW])


def test_dw_noisy_tfim_n13_two_steps_match_the_kraus_oracle():
    # the density-matrix benchmark's circuit at full size, two Trotter steps,
    # against the stored Kraus-form oracle values (tests/golden/make_dm_n13_golden.py)
    import os
    n = 13
    gold = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dm_noisy_tfim_n13.npz"))
    gates, noise = inputs.dm_noisy_tfim(n, 2)
    tfim = inputs.tfim_terms(n)
    with State(L.DM, n, L.F64) as st, Plan(L.DM, n, gates, L.F64, noise, flags=L.PLAN_DW) as p:
        st.run(p)
        z = st.expect(inputs.z_terms(n))
        t = st.expect(tfim)
        pr = st.probs(noise["readout_e"])
        rho = st.copy()
        tr = st.norm()
    errs = dict(z=maxerr(z, gold["z2"]), terms=maxerr(t, gold["tfim2"]),
                rho=maxerr(rho[gold["r"], gold["c"]], gold["rho2"]), probs=maxerr(pr, gold["probs2"]))
    print(f"dw dm n=13 two steps: {errs}")
    assert max(errs.values()) <= 1e-12
    assert tr == 1.0  # the identity coefficient is carried exactly


def test_dw_tfim_chain_matches_free_fermions():
    # a long chain at the depth of the large-state workload, against exact values
    from oracle import tfim_fermion
    n = 24
    gates, h = inputs.large_sv_tfim(n, 10)
    ref = tfim_fermion.tfim_observables(n, gates)
    with Plan(L.SV, n, gates, L.F64, flags=L.PLAN_DW) as p, State(L.SV, n, L.F64) as st:
        st.run(p)
        zz = np.real(st.expect(inputs.zz_terms(n)))
        x = np.real(st.expect(inputs.x_terms(n)))
        nrm = st.norm()
    err = max(maxerr(zz, ref["zz"]), maxerr(x, ref["x"]))
    print(f"dw tfim n={n}: max term error {err:.3e}, norm-1 {nrm - 1:.2e}")
    assert err <= 1e-12
    assert abs(nrm - 1) <= 1e-12


# ---------------------------------------------------------------- double-word residency
# A library-owned FP64 state keeps the double-word layout a double-word plan run
# leaves (no conversion back); reset keeps it, full-tile expectation passes read it
# as it is, and every other reader or plan converts it back first.

def test_resident_layout_through_reset_runs_expectations_and_copies():
    n = 18  # the double-word kernels take states of >= 18 index bits
    gates = inputs.large_sv_tfim(n, 3)[0]
    terms = inputs.tfim_terms(n) + inputs.z_terms(n) + inputs.random_pauli_terms(n, 20, 61)
    wide = [((1 << n) - 1, 0, 1.0), ((1 << n) - 1 ^ 0x3, (1 << n) - 1, -0.5)]  # X wider than a tile
    ref = oracle.sv_run(n, gates)
    eref = oracle.sv_expect(ref, n, terms)
    with State(L.SV, n, L.F64) as st, Plan(L.SV, n, gates, L.F64, flags=L.PLAN_DW) as p, \
            Plan(L.SV, n, gates, L.F64, flags=L.PLAN_FP64) as q:
        for rep in range(3):  # the second and third runs start from a reset in the double-word layout
            st.reset()
            st.run(p)
            assert p.last_run_dw()
            assert maxerr(st.expect(terms), eref) <= 1e-12, rep              # read in the double-word layout
            assert abs(st.expect(terms, sum=True, normalize=True) - oracle.energy(eref, terms)) <= 1e-11
        assert maxerr(st.copy(), ref) <= 1e-12                               # converted back for the copy
        st.run(p)                                                            # twice the circuit, from FP64
        ref2 = oracle.sv_run(n, gates, ref)
        assert maxerr(st.expect(wide), oracle.sv_expect(ref2, n, wide)) <= 1e-12  # general kernel: back to FP64
        st.reset()
        st.run(p)
        st.run(q)                                                            # FP64-pipe plan after a resident run
        assert maxerr(st.copy(), ref2) <= 1e-12
        st.reset()
        st.run(p)
        probs = st.probs(0.0)
        assert maxerr(probs, np.abs(ref) ** 2) <= 1e-12
        st.reset()
        st.run(p)
        out = np.zeros(len(terms))
        arr = L.encode_terms(terms)
        import ctypes
        L.check(L.lib().nwq_expect_pauli_sum_noalloc(st.h, arr, len(terms),
                                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                     L.EXPECT_TERMS))
        assert maxerr(out, eref) <= 1e-12
        st.load(ref2)                                                        # a load replaces the layout
        assert maxerr(st.copy(), ref2) <= 1e-15


def test_caller_owned_buffers_hold_fp64_after_double_word_runs():
    import torch
    n = 18
    gates = inputs.large_sv_tfim(n, 2)[0]
    t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    with State(L.SV, n, L.F64, buf=t.data_ptr(), buf_bytes=t.numel() * 16) as st, \
            Plan(L.SV, n, gates, L.F64, flags=L.PLAN_DW) as p:
        st.run(p)
        st.sync()
        assert p.last_run_dw()
        assert maxerr(t.cpu().numpy(), oracle.sv_run(n, gates)) <= 1e-12    # the caller's bytes are FP64


def test_resident_density_matrix_readers():
    n = 9  # 18 index bits
    gates, noise = inputs.dm_noisy_tfim(n, 3)
    terms = inputs.tfim_terms(n) + inputs.z_terms(n)
    rho = oracle.dm_run(n, gates, noise)
    with State(L.DM, n, L.F64) as st, Plan(L.DM, n, gates, L.F64, noise, flags=L.PLAN_DW) as p:
        for _ in range(2):
            st.reset()
            st.run(p)
            assert p.last_run_dw()
            assert maxerr(st.expect(terms), oracle.dm_expect(rho, n, terms)) <= 1e-12
            st.run(p)
            rho2 = oracle.dm_run(n, gates, noise, rho0=rho)
            assert maxerr(st.probs(0.02), oracle.dm_probs(rho2, n, 0.02)) <= 1e-12
            st.run(p)
            pa = st.pauli()
            st.load_pauli(pa)
            assert maxerr(st.pauli(), pa) == 0.0


def test_resident_reads_and_repeated_runs_keep_fp64_accuracy():
    # the sweeps' multiply-adds leave the low float of each pair unnormalised, and a
    # product of two such pairs would drop a term that is then not negligible: expectation
    # passes over a resident state renormalise every pair (exactly) before any product, and a
    # state kept resident from run to run is renormalised before the next run.  Against the
    # exact free-fermion values of the TFIM chain (reading the pairs unnormalised gave
    # 2.6e-13 here, the FP64 layout 3e-14)
    from oracle import tfim_fermion
    n = 22
    gates, h = inputs.large_sv_tfim(n, 10)
    zzt, xt = inputs.zz_terms(n), inputs.x_terms(n)

    def err(st, ref):
        zz, x = st.expect(zzt), st.expect(xt)
        return max(float(np.max(np.abs(zz - ref["zz"]))), float(np.max(np.abs(x - ref["x"]))))

    ref1 = tfim_fermion.tfim_observables(n, gates)
    with State(L.SV, n, L.F64) as st, Plan(L.SV, n, gates, L.F64, flags=L.PLAN_DW) as p:
        st.run(p)
        assert p.last_run_dw()
        e_resident = err(st, ref1)
        st.copy()
        e_fp64 = err(st, ref1)
        assert e_resident <= 1e-13 and e_fp64 <= 1e-13, (e_resident, e_fp64)
        st.reset()
        for _ in range(3):  # resident from run to run
            st.run(p)
        assert err(st, tfim_fermion.tfim_observables(n, gates * 3)) <= 1e-13
