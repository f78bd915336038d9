"""Host-side pin of the sweep planner of state vectors (no GPU): the merged
operators of a plan, applied in the plan's execution order as plain matrices,
reproduce the oracle's gate-by-gate state, for every plan form and shape."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim
from tests.dense import apply_local


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2401_06861_gb300 import build
    build.build()
    oracle.build()


def run_ops(n, ops, psi0):
    psi = psi0.copy()
    for qs, U in ops:
        psi = apply_local(psi, n, qs, U)
    return psi


@pytest.mark.parametrize("flags", [L.PLAN_FUSED, L.PLAN_NO_MERGE, L.PLAN_PLAIN])
@pytest.mark.parametrize("dtype", [L.F64, L.F32])
@pytest.mark.parametrize("n", [3, 8, 13])
def test_plan_operators_reproduce_oracle(n, dtype, flags):
    gates = inputs.random_circuit(n, 150, 7000 + n)
    psi0 = inputs.random_state(n, 7100 + n)
    with sim.Plan(L.SV, n, gates, dtype, flags=flags) as pl:
        ops = pl.ops()
        info = pl.info()
        _, og, on = pl.layout()
    assert len(ops) == info["ops"] and sum(on) == len(gates)
    if flags == L.PLAN_PLAIN:
        assert len(ops) == len(gates)
    assert np.max(np.abs(run_ops(n, ops, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


@pytest.mark.parametrize("tuning", [dict(tile_bits=10, fusion_bits=3, register_bits=3),
                                    dict(tile_bits=13, fusion_bits=4, register_bits=4), dict(fusion_bits=2)])
def test_tuned_plan_shapes_reproduce_oracle(tuning):
    n = 14
    gates, _ = inputs.large_sv_tfim(n, 4)
    gates = gates + inputs.random_circuit(n, 60, 7200)
    psi0 = inputs.random_state(n, 7300)
    with sim.Plan(L.SV, n, gates, L.F32, tuning=tuning) as pl:
        ops = pl.ops()
    assert np.max(np.abs(run_ops(n, ops, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


def test_tfim_bonds_merge_into_diagonal_operators():
    n = 12
    gates, _ = inputs.large_sv_tfim(n, 2)
    with sim.Plan(L.SV, n, gates, L.F64) as pl:
        ops = pl.ops()
    diag = [np.count_nonzero(U - np.diag(np.diag(U))) == 0 for _, U in ops]
    assert len(ops) < len(gates) and any(diag)
    psi0 = inputs.random_state(n, 3)
    assert np.max(np.abs(run_ops(n, ops, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


def test_ops_hook_refuses_other_plans():
    with sim.Plan(L.SV, 12, [("H", (0,), ())], L.F32, flags=L.PLAN_TC) as pl:
        with pytest.raises(L.NwqError):
            pl.ops()


@pytest.mark.parametrize("dtype", [L.F64, L.F32])
@pytest.mark.parametrize("n,family", [(8, "diag"), (13, "diag"), (16, "tfim"), (13, "mixed")])
def test_commuting_plans_reproduce_oracle(n, family, dtype):
    # NWQ_PLAN_COMMUTE: diagonal operators pass skipped diagonal operators
    if family == "diag":
        gates = inputs.random_circuit(n, 200, 7400 + n, names=["RZ", "CZ", "RZZ", "T", "P", "S", "RX", "H", "CX"],
                                      two_qubit_frac=0.5)
    elif family == "tfim":
        gates = inputs.large_sv_tfim(n, 6)[0]
    else:
        gates = inputs.random_circuit(n, 150, 7500 + n)
    psi0 = inputs.random_state(n, 7600 + n)
    with sim.Plan(L.SV, n, gates, dtype, flags=L.PLAN_COMMUTE) as pl:
        ops = pl.ops()
        _, _, on = pl.layout()
        pl.verify()
    assert sum(on) == len(gates)
    assert np.max(np.abs(run_ops(n, ops, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


def test_commuting_plans_need_fewer_sweeps_for_diagonal_bonds():
    # the depth-10 chain at n = 34: CX RZ CX bonds merge into diagonal
    # operators, which now share sweeps across Trotter steps
    gates, _ = inputs.large_sv_tfim(34, 10)
    with sim.Plan(L.SV, 34, gates, L.F32, flags=L.PLAN_NO_COMMUTE) as a, \
            sim.Plan(L.SV, 34, gates, L.F32, flags=L.PLAN_COMMUTE) as b, sim.Plan(L.SV, 34, gates, L.F32) as c:
        assert c.info()["sweeps"] == b.info()["sweeps"]  # commuting is the default
        ia, ib = a.info(), b.info()
    assert ib["ops"] == ia["ops"] and ib["fma_per_elem"] == ia["fma_per_elem"]
    assert ib["sweeps"] <= 0.6 * ia["sweeps"]


def pauli_coefficients(rho, n):
    """r[x + 2^n z] = Tr(rho P(x, z)), P(x, z) = i^{|x & z|} X^x Z^z (from the definition)."""
    N = 1 << n
    b = np.arange(N)
    popc = np.vectorize(lambda v: bin(int(v)).count("1"))
    r = np.zeros(N * N)
    for z in range(N):
        sign = (-1.0) ** popc(b & z)
        for x in range(N):
            v = (1j ** bin(x & z).count("1")) * np.sum(rho[b, b ^ x] * sign)
            r[x + N * z] = v.real
    return r


@pytest.mark.parametrize("flags", [L.PLAN_FUSED, L.PLAN_NO_MERGE, L.PLAN_PLAIN, L.PLAN_NO_RESCALE])
@pytest.mark.parametrize("dtype", [L.F64, L.F32])
@pytest.mark.parametrize("n", [2, 4])
def test_dm_plan_operators_reproduce_kraus_oracle(n, dtype, flags):
    # the density-matrix planner (gate + depolarising + relaxation lowered to
    # Pauli-transfer operators, merged, rescaled, grouped): its operators,
    # applied to the coefficients of |0..0><0..0|, give the Pauli coefficients
    # of the Kraus-form oracle's density matrix
    gates = inputs.random_circuit(n, 40, 7700 + n)
    noise = inputs.noise_params(n, seed=7800 + n)
    with sim.Plan(L.DM, n, gates, dtype, noise, flags=flags) as pl:
        ops = pl.ops()
        _, _, on = pl.layout()
    assert sum(on) == len(gates)
    N = 1 << n
    r = np.zeros(N * N, complex)
    r[N * np.arange(N)] = 1.0  # Tr(|0><0| X^x Z^z) = [x = 0]
    for bits, M in ops:
        assert np.max(np.abs(M.imag)) == 0.0
        r = apply_local(r, 2 * n, bits, M)
    ref = pauli_coefficients(oracle.dm_run(n, gates, noise), n)
    assert np.max(np.abs(r.imag)) == 0.0
    assert np.max(np.abs(r.real - ref)) <= 1e-12


def _deposit(v, S):
    out, i = 0, 0
    for b in range(64):
        if (S >> b) & 1:
            if (v >> i) & 1:
                out |= 1 << b
            i += 1
    return out


def _expect_terms(n, nt, seed):
    # Z strings, X/Y on low qubits, on high qubits, and wide X supports
    rng = np.random.default_rng(seed)
    terms = []
    for t in range(nt):
        kind = t % 4
        if kind == 0:
            x = 0
        elif kind == 1:
            x = int(rng.integers(1, 1 << min(n, 12)))
        elif kind == 2:
            qs = rng.choice(n, size=min(n, 3), replace=False)
            x = int(sum(1 << int(q) for q in qs))
        else:
            qs = rng.choice(n, size=min(n, 14), replace=False)
            x = int(sum(1 << int(q) for q in qs))
        z = int(rng.integers(0, 1 << n))
        terms.append((x, z, float(rng.normal())))
    return terms


@pytest.mark.parametrize("n", [3, 12, 20, 30])
@pytest.mark.parametrize("normalize", [False, True])
def test_expectation_pass_plan_invariants(n, normalize):
    terms = _expect_terms(n, 300, 900 + n)
    plan = sim.expect_plan(n, terms, normalize)
    T = min(n, 12)
    seen = {}
    for p, (tile, recs) in enumerate(plan["passes"]):
        assert bin(tile).count("1") == T and tile < (1 << n) and 0 < len(recs) <= 256
        m = 0
        while (tile >> m) & 1:
            m += 1
        assert m >= min(T, 4)  # contiguous low bits
        for out, xl, zl, zh, y in recs:
            seen[out] = seen.get(out, 0) + 1
            x, z = (0, 0) if out == len(terms) else (terms[out][0], terms[out][1])
            assert _deposit(xl, tile) == x and x & ~tile == 0  # X support inside the tile
            assert _deposit(zl, tile) | zh == z and zh & tile == 0
            assert y == bin(x & z).count("1") % 4
            if out == len(terms):  # the identity string rides with the low-tile terms
                assert normalize and tile == (1 << T) - 1
    for t in plan["general"]:
        seen[t] = seen.get(t, 0) + 1
        assert bin(terms[t][0] & ~0xF).count("1") > T - 4  # no tile can hold its X support
    want = set(range(len(terms))) | ({len(terms)} if normalize else set())
    assert set(seen) == want and all(v == 1 for v in seen.values())
    if n >= 20:
        assert plan["general"]  # the wide X supports take the general kernel
