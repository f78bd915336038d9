"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 path 1e-12 max absolute amplitude / density-matrix entry
error; FP32 path 1e-5 amplitude error and 1e-6 relative energy error, where
the relative energy error is |E - E_ref| / max(|E_ref|, ||H||_1) with
||H||_1 the sum of |coefficients| (random-parameter energies can be ~0).
"""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.sim import Plan, State

pytestmark = pytest.mark.gpu

TOL = {L.F64: 1e-12, L.F32: 1e-5}
DTYPES = [L.F64, L.F32]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    torch.cuda.init()
    yield


def maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


def rel_energy(e, eref, terms):
    return abs(e - eref) / max(abs(eref), sum(abs(t[2]) for t in terms))


# ------------------------------------------------------------------ state vector
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("flags", [L.PLAN_FUSED, L.PLAN_PLAIN, L.PLAN_NO_MERGE])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 13, 16])
def test_sv_random_circuits(n, flags, dtype):
    gates = inputs.random_circuit(n, 120 if n <= 13 else 60, 1000 + n)
    psi0 = inputs.random_state(n, 2000 + n)
    with State(L.SV, n, dtype) as st:
        st.load(psi0)
        st.apply(gates, flags=flags)
        got = st.copy()
    ref = oracle.sv_run(n, gates, psi0)
    err = maxerr(got, ref)
    print(f"sv n={n} flags={flags} dtype={dtype} max_abs_err={err:.3e}")
    assert err <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,family", [(18, "random"), (19, "random_mat"), (20, "tfim"), (18, "hea"),
                                      (19, "no_merge")])
def test_sv_specialised_kernels(n, family, dtype):
    # states of >= 18 qubits run run-time compiled sweep kernels: against the
    # oracle and against the interpreted kernel on the same plan structure
    flags = 0
    if family == "random":
        gates = inputs.random_circuit(n, 300, 3000 + n, names=[g for g in inputs.GATE_NAMES if not g.startswith("MAT")])
    elif family == "random_mat":
        gates = inputs.random_circuit(n, 150, 3100 + n)
    elif family == "tfim":
        gates = inputs.large_sv_tfim(n, 4)[0]
    elif family == "hea":
        gates = inputs.hea_ansatz(n, 4, inputs.hea_params(n, 4, 1)[0])[0]
    else:
        gates, flags = inputs.random_circuit(n, 120, 3200 + n), L.PLAN_NO_MERGE
    psi0 = inputs.random_state(n, 2100 + n)
    out = {}
    for extra in (0, L.PLAN_INTERPRETED):
        # a reusable plan compiles its kernels before its first run; FP64
        # plans take the FP64-pipe kernels here (the double-word ones round
        # differently; tests/test_gpu_dw.py checks them against the oracle)
        with State(L.SV, n, dtype) as st, Plan(L.SV, n, gates, dtype, flags=flags | extra | L.PLAN_FP64) as plan:
            st.load(psi0)
            st.run(plan)
            out[extra] = st.copy()
    ref = oracle.sv_run(n, gates, psi0)
    err, err_i = maxerr(out[0], ref), maxerr(out[0], out[L.PLAN_INTERPRETED])
    print(f"sv n={n} {family} dtype={dtype} specialised err {err:.3e}, vs interpreted {err_i:.3e}")
    assert err <= TOL[dtype]
    assert err_i <= (1e-14 if dtype == L.F64 else 1e-6)


@pytest.mark.parametrize("kind,dtype", [(L.SV, L.F32), (L.SV, L.F64), (L.DM, L.F64), (L.DM, L.F32)])
def test_autotuned_plan_shapes_all_agree_with_the_oracle(kind, dtype):
    from paper_2401_06861_gb300.sim import autotune
    if kind == L.SV:
        n = 19
        gates = inputs.random_circuit(n, 150, 4000, names=[g for g in inputs.GATE_NAMES if not g.startswith("MAT")])
        noise, ref = None, oracle.sv_run(n, gates)
    else:
        n = 9
        gates, noise = inputs.random_circuit(n, 80, 4100), inputs.noise_params(n, seed=4101)
        ref = oracle.dm_run(n, gates, noise)
    with State(kind, n, dtype) as st:
        res = autotune(st, gates, noise, reps=2)
        timed = [(t, ms) for t, ms in res["tried"] if ms >= 0]
        assert len(timed) == len(res["tried"]) >= 4
        assert res["best_ms"] == min(ms for _, ms in timed)
        for t, _ in res["tried"]:  # every candidate shape computes the same state
            with Plan(kind, n, gates, dtype, noise, tuning=t) as plan:
                st.reset()
                st.run(plan)
                got = st.copy()
            err = maxerr(got, ref)
            assert err <= (TOL[dtype] if kind == L.SV else (1e-12 if dtype == L.F64 else 1e-5)), (t, err)
    print(f"autotune kind={kind} dtype={dtype}: best {res['best']} {res['best_ms']:.3f} ms of {len(timed)}")


@pytest.mark.parametrize("dtype", DTYPES)
def test_sv_every_gate_on_every_qubit_position(dtype):
    # each gate kind on low, tile-boundary and top qubits of a 15-qubit state
    n = 15
    rng = np.random.default_rng(5)
    gates = []
    for name in inputs.GATE_NAMES:
        for q in (0, 2, 3, 4, 11, 12, 13, 14):
            if name in inputs.TWO_QUBIT:
                for q2 in (0, 3, 12, 14):
                    if q2 != q:
                        prm = inputs.random_unitary(4, rng) if name == "MAT2" else tuple(rng.uniform(-3, 3, inputs.N_PARAMS.get(name, 0)))
                        gates.append(inputs.gate(name, (q, q2), prm))
            else:
                prm = inputs.random_unitary(2, rng) if name == "MAT1" else tuple(rng.uniform(-3, 3, inputs.N_PARAMS.get(name, 0)))
                gates.append(inputs.gate(name, (q,), prm))
    psi0 = inputs.random_state(n, 77)
    ref = oracle.sv_run(n, gates, psi0)
    for flags in (L.PLAN_FUSED, L.PLAN_PLAIN):
        with State(L.SV, n, dtype) as st:
            st.load(psi0)
            st.apply(gates, flags=flags)
            err = maxerr(st.copy(), ref)
        print(f"all-gates n={n} flags={flags} dtype={dtype} ({len(gates)} gates) max_abs_err={err:.3e}")
        assert err <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_tfim_n10_40_steps(dtype):
    n = 10
    gates = inputs.tfim_trotter(n, 1.0, 1.0, 0.05, 40)
    terms = inputs.tfim_terms(n, 1.0, 1.0)
    ref = oracle.sv_run(n, gates)
    zref = oracle.sv_expect(ref, n, inputs.z_terms(n))
    eref = oracle.energy(oracle.sv_expect(ref, n, terms), terms)
    with State(L.SV, n, dtype) as st:
        st.apply(gates)
        psi = st.copy()
        z = st.expect(inputs.z_terms(n), normalize=True)
        e = st.expect(terms, sum=True, normalize=True)
        e_raw = st.expect(terms, sum=True)
        nrm = st.norm()
    aerr, zerr, rerr = maxerr(psi, ref), maxerr(z, zref), rel_energy(e, eref, terms)
    print(f"tfim n=10 dtype={dtype}: amp {aerr:.3e}  <Z> {zerr:.3e}  rel energy {rerr:.3e} "
          f"(unnormalised {rel_energy(e_raw, eref, terms):.3e}, norm-1 {nrm - 1:.3e})")
    assert aerr <= TOL[dtype]
    assert zerr <= TOL[dtype]
    assert rerr <= (1e-12 if dtype == L.F64 else 1e-6)
    assert abs(nrm - 1) <= (1e-13 if dtype == L.F64 else 1e-4)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 4, 7, 8, 11, 12, 13, 15, 17])
def test_sv_expectations(n, dtype):
    psi0 = inputs.random_state(n, 300 + n)
    terms = inputs.random_pauli_terms(n, 40, 400 + n) + inputs.z_terms(n) + inputs.x_terms(n)
    ref = oracle.sv_expect(psi0, n, terms)
    with State(L.SV, n, dtype) as st:
        st.load(psi0)
        got = st.expect(terms)
        tot = st.expect(terms, sum=True)
        totn = st.expect(terms, sum=True, normalize=True)
        gotn = st.expect(terms, normalize=True)
    tol = 1e-12 if dtype == L.F64 else 2e-6
    assert maxerr(got, ref) <= tol
    assert abs(tot - oracle.energy(ref, terms)) <= tol * len(terms)
    assert maxerr(gotn, ref) <= tol and abs(totn - oracle.energy(ref, terms)) <= tol * len(terms)


def _wide_terms(n, rng):
    """Strings whose X support spans many high bits (some wider than any
    shared-memory tile), with Y factors, the identity and a duplicate."""
    full = (1 << n) - 1
    t = [(full, 0, 0.5), (full, full, -0.25), (full & 0xAAAAAAAAA, full & 0x555555555, 0.75), (0, 0, 1.5)]
    for w in (5, 8, 9, 11, 12, 13):
        bits = rng.choice(np.arange(4, n), size=min(w, n - 4), replace=False)
        x = int(sum(1 << int(b) for b in bits)) | int(rng.integers(0, 16))
        t.append((x, int(rng.integers(0, 1 << n)), float(rng.uniform(-1, 1))))
    t.append(t[5])
    return t


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [13, 16, 18])
def test_sv_expectations_tile_passes(n, dtype):
    # terms spread over the low tile, several high-bit tiles and the general kernel
    rng = np.random.default_rng(500 + n)
    psi0 = inputs.random_state(n, 310 + n)
    terms = (inputs.random_pauli_terms(n, 30, 410 + n) + inputs.tfim_terms(n) + inputs.x_terms(n)
             + [(1 << (n - 1), 1, 1.0), ((1 << (n - 1)) | 1, (1 << (n - 1)) | 2, -1.0)] + _wide_terms(n, rng))
    ref = oracle.sv_expect(psi0, n, terms)
    with State(L.SV, n, dtype) as st:
        st.load(psi0)
        got = st.expect(terms)
        gotn = st.expect(terms, normalize=True)
        tot = st.expect(terms, sum=True, normalize=True)
    tol = 1e-12 if dtype == L.F64 else 2e-6
    assert maxerr(got, ref) <= tol
    assert maxerr(gotn, ref) <= tol
    assert abs(tot - oracle.energy(ref, terms)) <= tol * len(terms)


@pytest.mark.parametrize("dtype", DTYPES)
def test_sv_expectations_many_terms_one_pass(dtype):
    # more terms than one launch takes (256) inside the same tile
    n = 10
    psi0 = inputs.random_state(n, 320)
    terms = inputs.random_pauli_terms(n, 700, 420)
    ref = oracle.sv_expect(psi0, n, terms)
    with State(L.SV, n, dtype) as st:
        st.load(psi0)
        got = st.expect(terms)
        tot = st.expect(terms, sum=True)
    tol = 1e-12 if dtype == L.F64 else 2e-6
    assert maxerr(got, ref) <= tol
    assert abs(tot - oracle.energy(ref, terms)) <= tol * len(terms)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,e", [(1, 0.0), (1, 0.1), (6, 0.02), (14, 0.02), (14, 0.0)])
def test_sv_probs_with_readout(n, e, dtype):
    psi0 = inputs.random_state(n, 50 + n)
    with State(L.SV, n, dtype) as st:
        st.load(psi0)
        got = st.probs(e)
    ref = oracle.sv_probs(psi0, n, e)
    tol = 1e-14 if dtype == L.F64 else 1e-6
    assert maxerr(got, ref) <= tol


def test_sv_caller_owned_buffer_and_stream():
    import torch
    n = 14
    buf = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    gates = inputs.random_circuit(n, 50, 9)
    with State(L.SV, n, L.F64, buf=buf.data_ptr(), buf_bytes=buf.numel() * 16, stream=s.cuda_stream) as st:
        st.apply(gates)
        st.sync()
        got = buf.cpu().numpy()
    assert maxerr(got, oracle.sv_run(n, gates)) <= 1e-12


# ------------------------------------------------------------------ density matrix
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("flags", [L.PLAN_FUSED, L.PLAN_PLAIN, L.PLAN_NO_MERGE, L.PLAN_NO_RESCALE])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_dm_random_noisy_circuits(n, flags, dtype):
    gates = inputs.random_circuit(n, 60, 3000 + n)
    noise = inputs.noise_params(n, seed=40 + n)
    rho0 = inputs.random_density(n, 4000 + n)
    with State(L.DM, n, dtype) as st:
        st.load(rho0)
        st.apply(gates, noise, flags)
        got = st.copy()
    ref = oracle.dm_run(n, gates, noise, rho0)
    err = maxerr(got, ref)
    print(f"dm n={n} flags={flags} dtype={dtype} max_abs_err={err:.3e}")
    assert err <= TOL[dtype]


@pytest.mark.parametrize("variant", ["rz_virtual", "depol_pauli_form", "noiseless"])
def test_dm_noise_variants(variant):
    n = 4
    gates = inputs.random_circuit(n, 50, 7)
    noise = None if variant == "noiseless" else inputs.noise_params(n, seed=3, **{variant: True})
    rho0 = inputs.random_density(n, 8)
    with State(L.DM, n, L.F64) as st:
        st.load(rho0)
        st.apply(gates, noise)
        got = st.copy()
    assert maxerr(got, oracle.dm_run(n, gates, noise, rho0)) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
def test_dm_init_load_copy_roundtrip(dtype):
    n = 6
    with State(L.DM, n, dtype) as st:
        assert maxerr(st.copy(), oracle.dm_zero(n)) == 0.0
        rho = inputs.random_density(n, 1)
        st.load(rho)
        assert maxerr(st.copy(), rho) <= (1e-15 if dtype == L.F64 else 1e-7)


@pytest.mark.parametrize("dtype", DTYPES)
def test_dm_noisy_tfim_n8_20_steps(dtype):
    n = 8
    gates, noise = inputs.dm_noisy_tfim(n, 20)
    terms = inputs.tfim_terms(n)
    ref = oracle.dm_run(n, gates, noise)
    with State(L.DM, n, dtype) as st:
        st.apply(gates, noise)
        rho = st.copy()
        z = st.expect(inputs.z_terms(n))
        e = st.expect(terms, sum=True)
        p = st.probs(noise["readout_e"])
    zref = oracle.dm_expect(ref, n, inputs.z_terms(n))
    eref = oracle.energy(oracle.dm_expect(ref, n, terms), terms)
    pref = oracle.dm_probs(ref, n, noise["readout_e"])
    print(f"dm tfim n=8 dtype={dtype}: rho {maxerr(rho, ref):.3e} <Z> {maxerr(z, zref):.3e} "
          f"rel E {rel_energy(e, eref, terms):.3e} probs {maxerr(p, pref):.3e}")
    assert maxerr(rho, ref) <= TOL[dtype]
    assert rel_energy(e, eref, terms) <= (1e-12 if dtype == L.F64 else 1e-6)
    assert maxerr(p, pref) <= (1e-14 if dtype == L.F64 else 1e-6)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_dm_expectations_and_probs(n):
    rho0 = inputs.random_density(n, 90 + n)
    terms = inputs.random_pauli_terms(n, 30, 91 + n)
    with State(L.DM, n, L.F64) as st:
        st.load(rho0)
        got = st.expect(terms)
        assert maxerr(st.expect(terms, normalize=True), got) <= 1e-14
        assert abs(st.norm() - 1) <= 1e-14
        for e in (0.0, 0.02, 0.25):
            assert maxerr(st.probs(e), oracle.dm_probs(rho0, n, e)) <= 1e-14
    assert maxerr(got, oracle.dm_expect(rho0, n, terms)) <= 1e-14


# ------------------------------------------------------------------ full-size density matrix (n = 13)
def test_dm_n13_noiseless_matches_sv_oracle_outer_product():
    n = 13
    gates = inputs.tfim_trotter(n, 1.0, 1.0, 0.05, 2)
    psi = oracle.sv_run(n, gates)
    terms = inputs.random_pauli_terms(n, 60, 5) + inputs.tfim_terms(n)
    with State(L.DM, n, L.F64) as st:
        st.apply(gates)
        got = st.expect(terms)
        rho = st.copy()
    assert maxerr(got, oracle.sv_expect(psi, n, terms)) <= 1e-12
    rng = np.random.default_rng(1)
    r = rng.integers(0, 1 << n, 4000)
    c = rng.integers(0, 1 << n, 4000)
    assert maxerr(rho[r, c], psi[r] * psi[c].conj()) <= 1e-12


def _golden_n13():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dm_noisy_tfim_n13.npz")
    return np.load(path)


@pytest.mark.parametrize("dtype", DTYPES)
def test_dm_n13_noisy_tfim_steps_match_the_kraus_oracle(dtype):
    # The density-matrix benchmark's noisy entangling circuit at its full
    # size (paper Sec. III: TFIM chain with depolarising and relaxation after
    # every gate), against the Kraus-form oracle (tests/golden/
    # make_dm_n13_golden.py): one Trotter step through the one-shot call, two
    # steps through a reusable plan (the specialised kernels the benchmark
    # runs); every <Z_i>, all 25 TFIM terms, 10^4 sampled rho entries and
    # the readout-noisy outcome distribution.
    n = 13
    gold = _golden_n13()
    r, c = gold["r"], gold["c"]
    tfim = inputs.tfim_terms(n)
    ro = inputs.noise_params(n)["readout_e"]
    tol = TOL[dtype]

    def check(st, k):
        z = st.expect(inputs.z_terms(n))
        t = st.expect(tfim)
        e = st.expect(tfim, sum=True)
        p = st.probs(ro)
        rho = st.copy()
        eref = oracle.energy(gold[f"tfim{k}"], tfim)
        errs = dict(z=maxerr(z, gold[f"z{k}"]), terms=maxerr(t, gold[f"tfim{k}"]),
                    rho=maxerr(rho[r, c], gold[f"rho{k}"]), probs=maxerr(p, gold[f"probs{k}"]),
                    rel_energy=rel_energy(e, eref, tfim))
        print(f"dm n=13 noisy TFIM, {k} step(s), dtype={dtype}: {errs}")
        assert errs["z"] <= tol and errs["terms"] <= tol and errs["rho"] <= tol
        assert errs["probs"] <= (1e-12 if dtype == L.F64 else 1e-6)
        assert errs["rel_energy"] <= (1e-12 if dtype == L.F64 else 1e-6)

    gates1, noise = inputs.dm_noisy_tfim(n, 1)
    gates2, _ = inputs.dm_noisy_tfim(n, 2)
    with State(L.DM, n, dtype) as st:
        st.apply(gates1, noise)
        check(st, 1)
    with State(L.DM, n, dtype) as st, Plan(L.DM, n, gates2, dtype, noise) as plan:
        st.run(plan)
        check(st, 2)


def test_dm_n13_noisy_product_state_matches_single_qubit_oracle():
    # J = 0: no entangling gates, so rho is a product of one-qubit states,
    # each given by the oracle on one qubit with that qubit's T1/T2.
    n, steps = 13, 20
    noise = inputs.noise_params(n)
    gates = inputs.tfim_trotter(n, 0.0, 1.0, 0.05, steps)
    gates = [g for g in gates if g[0] != "RZ" and g[0] != "CX"]
    z1 = []
    for q in range(n):
        nq = dict(noise, T1_us=noise["T1_us"][q:q + 1], T2_us=noise["T2_us"][q:q + 1])
        g1 = [(name, (0,), prm) for name, (qq,), prm in gates if qq == q]
        r1 = oracle.dm_run(1, g1, nq)
        z1.append(oracle.dm_expect(r1, 1, [(0, 1, 1.0)])[0])
    z1 = np.array(z1)
    pairs = [(0, (1 << i) | (1 << j), 1.0) for i, j in [(0, 1), (3, 9), (5, 12)]]
    with State(L.DM, n, L.F64) as st:
        st.apply(gates, noise)
        z = st.expect(inputs.z_terms(n))
        zz = st.expect(pairs)
    assert maxerr(z, z1) <= 1e-12
    assert maxerr(zz, [z1[0] * z1[1], z1[3] * z1[9], z1[5] * z1[12]]) <= 1e-12


def test_dm_n13_bench_config_plans_agree_and_are_physical():
    from scipy.sparse.linalg import eigsh
    from scipy import sparse
    n = 13
    gates, noise = inputs.dm_noisy_tfim(n, 20)
    terms = inputs.tfim_terms(n)
    out = {}
    for key, dtype, flags in (("fused64", L.F64, 0), ("plain64", L.F64, L.PLAN_PLAIN), ("fused32", L.F32, 0)):
        with State(L.DM, n, dtype) as st:
            st.apply(gates, noise, flags)
            out[key] = (st.pauli().astype(np.float64), st.expect(inputs.z_terms(n)), st.expect(terms, sum=True),
                        st.probs(noise["readout_e"]))
    a, b, c = out["fused64"], out["plain64"], out["fused32"]
    assert a[0][0] == 1.0  # trace is preserved exactly
    assert maxerr(a[0], b[0]) <= 1e-12
    assert maxerr(a[0], c[0]) <= 1e-5
    assert rel_energy(c[2], a[2], terms) <= 1e-6
    assert abs(a[3].sum() - 1) <= 1e-12 and a[3].min() >= -1e-15
    # variational bound: a physical state cannot go below the ground energy
    N = 1 << n
    bb = np.arange(N)
    diag = -sum((1 - 2 * ((bb >> i) & 1)) * (1 - 2 * ((bb >> (i + 1)) & 1)) for i in range(n - 1)).astype(float)
    H = sparse.diags(diag).tocsr()
    for i in range(n):
        H = H + sparse.csr_matrix((-np.ones(N), (bb ^ (1 << i), bb)), shape=(N, N))
    e0 = eigsh(H, k=1, which="SA")[0][0]
    assert a[2] >= e0 - 1e-9


# ------------------------------------------------------------------ full-size state vector (128 GiB)
def _closed_form_rabi(n, h, dt, steps, idx):
    phi = 2 * h * dt * steps
    amp = np.ones(len(idx), complex)
    for i in range(n):
        bit = (idx >> i) & 1
        amp *= np.where(bit, -1j * np.sin(phi[i] / 2), np.cos(phi[i] / 2))
    return amp


@pytest.mark.parametrize("flags", [L.PLAN_FUSED, L.PLAN_NO_MERGE])
def test_sv_long_x_rotation_chains(flags):
    # 900 X-rotations with |tan| <= 1 between permutations and no diagonal:
    # complex128 plans carry their cos factors as one deferred scalar, which
    # must be re-applied whenever its exponent leaves range and at the end
    n = 10
    rng = np.random.default_rng(41)
    gates = []
    for i in range(900):
        q = int(rng.integers(n))
        gates.append(inputs.gate("RX", (q,), (float(rng.uniform(-1.5, 1.5)),)))
        if i % 3 == 2:
            gates.append(inputs.gate("CX", (q, (q + 1 + int(rng.integers(n - 1))) % n)))
    psi0 = inputs.random_state(n, 43)
    ref = oracle.sv_run(n, gates, psi0)
    for dtype in DTYPES:
        with State(L.SV, n, dtype) as st, Plan(L.SV, n, gates, dtype, flags=flags) as p:
            st.load(psi0)
            st.run(p)
            assert maxerr(st.copy(), ref) <= TOL[dtype]
            assert abs(st.norm() - np.sum(np.abs(ref) ** 2)) <= TOL[dtype]


@pytest.mark.parametrize("n,dtype", [(33, L.F64), (34, L.F32)])
def test_large_sv_rabi_closed_form(n, dtype):
    import torch
    rng = np.random.default_rng(n)
    h = rng.uniform(0.5, 2.0, n)
    steps = 1
    gates = [g for g in inputs.tfim_trotter(n, 0.0, h, 0.05, steps) if g[0] == "RX"]
    tdt = torch.complex128 if dtype == L.F64 else torch.complex64
    buf = torch.empty(1 << n, dtype=tdt, device="cuda")
    with State(L.SV, n, dtype, buf=buf.data_ptr(), buf_bytes=buf.numel() * buf.element_size()) as st:
        st.apply(gates)
        z = st.expect(inputs.z_terms(n)[:4] + inputs.z_terms(n)[-4:])
        idx = np.concatenate([rng.integers(0, 1 << n, 2000, dtype=np.int64), [0, (1 << n) - 1]])
        got = buf[torch.from_numpy(idx).cuda()].cpu().numpy()
    phi = 2 * h * 0.05 * steps
    assert maxerr(z, np.cos(np.concatenate([phi[:4], phi[-4:]]))) <= (1e-12 if dtype == L.F64 else 1e-5)
    assert maxerr(got, _closed_form_rabi(n, h, 0.05, steps, idx)) <= TOL[dtype]
    del buf
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,dtype", [(33, L.F64), (34, L.F32)])
def test_large_sv_tfim_matches_free_fermions(n, dtype):
    # the full-size depth-10 TFIM chains, run as the benchmark runs them (one
    # reusable fused plan), against exact free-fermion expectation values
    from oracle import tfim_fermion
    gates, h = inputs.large_sv_tfim(n, 10)
    ref = tfim_fermion.tfim_observables(n, gates)
    terms = inputs.tfim_terms(n, 1.0, h)
    eref = -float(np.sum(ref["zz"])) - float(np.dot(h, ref["x"]))
    norm = dtype == L.F32  # FP32: values of the renormalised state (the flagged option)
    with Plan(L.SV, n, gates, dtype) as p, State(L.SV, n, dtype) as st:
        st.run(p)
        zz = np.real(st.expect(inputs.zz_terms(n), normalize=norm))
        x = np.real(st.expect(inputs.x_terms(n), normalize=norm))
        z0 = float(np.real(st.expect([(0, 1, 1.0)], normalize=norm)[0]))
        e = st.expect(terms, sum=True, normalize=norm)
        nrm = st.norm()
    err = max(maxerr(zz, ref["zz"]), maxerr(x, ref["x"]), abs(z0 - ref["z0"]))
    print(f"n={n} dtype={dtype}: max term error {err:.3e}, E {e:.12f} vs {eref:.12f}, norm-1 {nrm - 1:.2e}")
    assert err <= TOL[dtype]
    assert rel_energy(e, eref, terms) <= (1e-12 if dtype == L.F64 else 1e-6)


def test_sv_n28_fp32_vs_fp64_tfim():
    n = 28
    gates, h = inputs.large_sv_tfim(n, steps=3)
    terms = inputs.tfim_terms(n, 1.0, h)
    res = {}
    for dtype in DTYPES:
        with State(L.SV, n, dtype) as st:
            st.apply(gates)
            res[dtype] = (st.expect(terms, sum=True), st.expect(inputs.z_terms(n)))
    rerr = rel_energy(res[L.F32][0], res[L.F64][0], terms)
    print(f"n=28 fp32 vs fp64: rel energy {rerr:.3e}, <Z> {maxerr(res[L.F32][1], res[L.F64][1]):.3e}")
    assert rerr <= 1e-6
    assert maxerr(res[L.F32][1], res[L.F64][1]) <= 1e-5


def test_sv_n33_complex64_amplitudes_vs_complex128():
    # amplitude-level FP32 error at full size: the depth-10 chain at n = 33 in
    # complex128 (128 GiB) and in complex64 (64 GiB), fused and tensor-core plans
    import torch
    n = 33
    gates, h = inputs.large_sv_tfim(n, 10)
    terms = inputs.tfim_terms(n, 1.0, h)
    ref = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    with State(L.SV, n, L.F64, buf=ref.data_ptr(), buf_bytes=ref.numel() * 16) as st, Plan(L.SV, n, gates, L.F64) as p:
        st.run(p)
        e_ref = st.expect(terms, sum=True)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    for flags in (L.PLAN_FUSED, L.PLAN_TC):
        with State(L.SV, n, L.F32, buf=psi.data_ptr(), buf_bytes=psi.numel() * 8) as st, \
                Plan(L.SV, n, gates, L.F32, flags=flags) as p:
            st.run(p)
            e = st.expect(terms, sum=True, normalize=True)
        torch.cuda.synchronize()
        err = max((psi[a:a + (1 << 27)].to(torch.complex128) - ref[a:a + (1 << 27)]).abs().max().item()
                  for a in range(0, 1 << n, 1 << 27))
        print(f"n=33 complex64 flags={flags}: max amplitude error {err:.3e}, rel energy {rel_energy(e, e_ref, terms):.3e}")
        assert err <= TOL[L.F32]
        assert rel_energy(e, e_ref, terms) <= 1e-6
    del ref, psi
    torch.cuda.empty_cache()


def test_qasm_program_on_the_gpu():
    from paper_2401_06861_gb300 import qasm
    prog = """OPENQASM 2.0;
    include "qelib1.inc";
    qreg q[5];
    gate layer(a) x, y { ry(a) x; rz(-a/2) y; cx x, y; }
    h q;
    layer(0.3) q[0], q[1];
    layer(1.1) q[3], q[4];
    cp(pi/5) q[1], q[2];
    crz(0.9) q[2], q[3];
    ch q[4], q[0];
    u3(0.2, 0.4, -0.6) q[2];
    rzz(0.25) q[0], q[4];
    """
    r = qasm.parse(prog)
    ref = oracle.sv_run(r["n"], r["gates"])
    for dtype in DTYPES:
        with State(L.SV, r["n"], dtype) as st:
            st.apply(r["gates"])
            assert maxerr(st.copy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("kind,dtype", [(L.SV, L.F64), (L.SV, L.F32), (L.DM, L.F64), (L.DM, L.F32)])
def test_checkpoint_and_resume_is_bit_exact(kind, dtype):
    # a run split at a circuit boundary, its state parked in host memory and
    # loaded into a fresh state, ends bit-identical to the run that took the same
    # checkpoint and went on.  Without the checkpoint an FP64 run keeps its
    # double-word layout between the two circuits (the checkpoint rounds it to
    # FP64 values), so the uninterrupted run agrees to the FP64 tolerance; FP32
    # runs keep one layout and agree bit for bit.
    n = 20 if kind == L.SV else 10
    g = inputs.random_circuit(n, 160, 4200, names=[x for x in inputs.GATE_NAMES if not x.startswith("MAT")])
    noise = inputs.noise_params(n, seed=4201) if kind == L.DM else None
    a, b = g[:90], g[90:]
    with Plan(kind, n, g, dtype, noise) as pf, Plan(kind, n, a, dtype, noise) as pa, \
            Plan(kind, n, b, dtype, noise) as pb:
        with State(kind, n, dtype) as st:
            st.run(pa)
            saved = st.copy() if kind == L.SV else st.pauli()
        with State(kind, n, dtype) as st:
            st.load(saved) if kind == L.SV else st.load_pauli(saved)
            st.run(pb)
            resumed = st.copy() if kind == L.SV else st.pauli()
        with State(kind, n, dtype) as st:
            st.run(pa)
            st.copy() if kind == L.SV else st.pauli()  # the checkpoint, taken and not used
            st.run(pb)
            straight = st.copy() if kind == L.SV else st.pauli()
        with State(kind, n, dtype) as st:
            st.run(pa)
            st.run(pb)
            uninterrupted = st.copy() if kind == L.SV else st.pauli()
    assert np.array_equal(resumed, straight)
    if dtype == L.F32:
        assert np.array_equal(resumed, uninterrupted)
    else:
        assert float(np.max(np.abs(resumed - uninterrupted))) <= 1e-13


def test_dm_maximum_size_n16_product_state():
    # the largest density matrix (4^16 FP64 Pauli coefficients, 32 GiB): a
    # product-state circuit with the full noise model against one-qubit oracles
    n = 16
    noise = inputs.noise_params(n, seed=4300)
    rng = np.random.default_rng(4301)
    gates = []
    for q in range(n):
        for name in ("RX", "RY", "RZ"):
            gates.append(inputs.gate(name, (q,), (float(rng.uniform(-np.pi, np.pi)),)))
    z1 = []
    for q in range(n):
        nq = dict(noise, T1_us=noise["T1_us"][q:q + 1], T2_us=noise["T2_us"][q:q + 1])
        r1 = oracle.dm_run(1, [(g[0], (0,), g[2]) for g in gates if g[1][0] == q], nq)
        z1.append(oracle.dm_expect(r1, 1, [(0, 1, 1.0)])[0])
    with State(L.DM, n, L.F64) as st:
        st.apply(gates, noise)
        z = st.expect(inputs.z_terms(n))
        tr = st.expect([(0, 0, 1.0)])[0]
    assert maxerr(z, z1) <= 1e-12
    assert abs(tr - 1.0) <= 1e-14


@pytest.mark.parametrize("kind,dtype", [(L.SV, L.F64), (L.SV, L.F32), (L.DM, L.F64), (L.DM, L.F32)])
def test_empty_circuits_and_term_lists(kind, dtype):
    # degenerate inputs: no gates (one-shot and planned), no terms
    n = 20 if kind == L.SV else 10
    with State(kind, n, dtype) as st, Plan(kind, n, [], dtype) as p:
        st.apply([])
        st.run(p)
        assert p.info()["sweeps"] == 0
        assert len(st.expect([])) == 0 and st.expect([], sum=True) == 0.0
        z = st.expect(inputs.z_terms(n), normalize=True)
        assert maxerr(z, np.ones(n)) <= 1e-6
        probs = st.probs()
        assert probs[0] == pytest.approx(1.0, abs=1e-6) and abs(probs.sum() - 1.0) <= 1e-6
