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
