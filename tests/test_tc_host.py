"""Tensor-core plans on the host (no GPU): the dense five-qubit blocks the
planner fuses, applied in order as plain matrices, reproduce the oracle's
gate-by-gate state; every block is unitary and accounts for its gates; the
tile geometry passes the plan checker; unsupported requests are refused."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2401_06861_gb300 import build
    build.build()
    oracle.build()


def apply_block(psi, n, qs, U):
    """psi <- U on qubits qs (local index bit i <-> qubit qs[i]), by index gathering."""
    others = [q for q in range(n) if q not in qs]
    r = np.arange(1 << (n - len(qs)))
    base = np.zeros_like(r)
    for i, q in enumerate(others):
        base |= ((r >> i) & 1) << q
    j = np.arange(1 << len(qs))
    off = np.zeros_like(j)
    for i, q in enumerate(qs):
        off |= ((j >> i) & 1) << q
    idx = base[:, None] | off[None, :]
    out = psi.copy()
    out[idx] = psi[idx] @ U.T
    return out


def run_blocks(n, blocks, psi0):
    psi = psi0.copy()
    for qs, U in blocks:
        psi = apply_block(psi, n, qs, U)
    return psi


@pytest.mark.parametrize("n,seed", [(12, 1), (12, 2), (13, 3), (14, 4)])
def test_blocks_reproduce_oracle_random_circuits(n, seed):
    gates = inputs.random_circuit(n, 80, seed)
    psi0 = inputs.random_state(n, seed + 100)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        blocks = pl.tc_blocks()
        pl.verify()
        sweeps, og, on = pl.layout()
    assert sum(on) == len(gates)
    assert sweeps == [1] * len(blocks)
    ref = oracle.sv_run(n, gates, psi0)
    got = run_blocks(n, blocks, psi0)
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_blocks_reproduce_oracle_tfim_chain():
    n = 16
    gates, _ = inputs.large_sv_tfim(n, 3)
    psi0 = inputs.random_state(n, 7)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        blocks = pl.tc_blocks()
        info = pl.info()
        pl.verify()
    assert info["sweeps"] == len(blocks) and info["ops"] == len(blocks)
    state_bytes = 8 * (1 << n)
    assert info["bytes"] == pytest.approx(2 * state_bytes * len(blocks))
    assert info["fma_per_elem"] == pytest.approx(384 * len(blocks))
    # fusion packs the 3 x (15 x 3 + 16) = 183 gates into far fewer passes: the
    # CX RZ CX bonds fold into diagonal gates, which pass one another
    assert len(blocks) <= 8
    ref = oracle.sv_run(n, gates, psi0)
    assert np.max(np.abs(run_blocks(n, blocks, psi0) - ref)) <= 1e-12


def test_blocks_are_unitary_on_valid_qubits():
    n = 13
    gates = inputs.random_circuit(n, 120, 11)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        blocks = pl.tc_blocks()
    for qs, U in blocks:
        assert len(qs) == 5 and list(qs) == sorted(set(qs)) and 0 <= qs[0] and qs[-1] < n
        assert np.max(np.abs(U @ U.conj().T - np.eye(32))) <= 1e-12


def test_edge_qubits_and_padding():
    # gates only on the top qubits and on qubit 0: padded blocks, tiles whose
    # block bits sit far above the row bits, and a block holding qubit 0
    n = 14
    gates = [("H", (13,), ()), ("CX", (13, 12), ()), ("RX", (11,), (0.3,)), ("CX", (0, 13), ()),
             ("MAT1", (9,), inputs.random_unitary(2, np.random.default_rng(5))), ("T", (0,), ())]
    psi0 = inputs.random_state(n, 9)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        blocks = pl.tc_blocks()
        pl.verify()
    assert np.max(np.abs(run_blocks(n, blocks, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


def test_empty_circuit_has_no_blocks():
    with sim.Plan(L.SV, 12, [], dtype=L.F32, flags=L.PLAN_TC) as pl:
        assert pl.info()["sweeps"] == 0
        assert pl.tc_blocks() == []


@pytest.mark.parametrize("kind,n,dtype", [(L.SV, 11, L.F32), (L.SV, 12, L.F64), (L.DM, 8, L.F32)])
def test_unsupported_requests(kind, n, dtype):
    with pytest.raises(L.NwqError) as e:
        sim.Plan(kind, n, [("H", (0,), ())], dtype=dtype, flags=L.PLAN_TC)
    assert e.value.code == L.EUNSUPPORTED


def test_not_a_tc_plan():
    with sim.Plan(L.SV, 12, [("H", (0,), ())], dtype=L.F32) as pl:
        with pytest.raises(L.NwqError):
            pl.tc_blocks()


def test_fusion_bits_5_is_the_tensor_core_plan():
    # the autotuner's shape for tensor-core plans: fusion_bits = 5
    n = 13
    gates = inputs.random_circuit(n, 60, 21)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as a, \
            sim.Plan(L.SV, n, gates, dtype=L.F32, tuning={"fusion_bits": 5}) as b:
        ba, bb = a.tc_blocks(), b.tc_blocks()
    assert [q for q, _ in ba] == [q for q, _ in bb]
    assert all(np.array_equal(x, y) for (_, x), (_, y) in zip(ba, bb))
    with pytest.raises(L.NwqError) as e:
        sim.Plan(L.SV, n, gates, dtype=L.F64, tuning={"fusion_bits": 5})
    assert e.value.code == L.EUNSUPPORTED


def _tf32_rna(x):
    """Round float32 values to TF32 (10 explicit mantissa bits), to nearest with ties away from zero."""
    u = np.asarray(x, np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def test_three_term_tf32_split_reaches_fp32_accuracy():
    # the tensor-core arithmetic, emulated: inputs split x = hi + lo with both
    # parts TF32, products lo*hi + hi*lo + hi*hi accumulated in FP32, against
    # the exact (FP64) 64-term real contraction of a random unitary's real form
    rng = np.random.default_rng(3)
    U = inputs.random_unitary(32, rng)
    M = np.block([[U.real, -U.imag], [U.imag, U.real]])  # acts on (re, im) halves
    X = (rng.standard_normal((64, 128)) * 1e-3).astype(np.float32)
    Mf = M.astype(np.float32)
    mh = _tf32_rna(Mf)
    ml = _tf32_rna(M - mh.astype(np.float64))
    xh = _tf32_rna(X)
    xl = _tf32_rna(X - xh)
    f32 = lambda a, b: (a.astype(np.float32) @ b.astype(np.float32)).astype(np.float64)
    D = f32(ml, xh) + f32(mh, xl) + f32(mh, xh)
    exact = M @ X.astype(np.float64)
    scale = np.abs(M) @ np.abs(X.astype(np.float64))
    rel = np.max(np.abs(D - exact) / scale)
    one_term = np.max(np.abs(f32(mh, xh) - exact) / scale)
    assert rel < 2.0 ** -19, rel          # FP32-level (a 64-term FP32 sum of exact products ~ 2^-20)
    assert one_term > 2.0 ** -14          # a single TF32 product is far coarser


def test_fusion_lets_diagonal_gates_pass_each_other():
    # the depth-10 chains of the large-state workloads: diagonal bond gates
    # commute, so blocks follow the light cone instead of one Trotter step each
    for n, most in [(26, 40), (34, 50)]:
        gates, _ = inputs.large_sv_tfim(n, 10)
        with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
            nb = pl.info()["sweeps"]
            _, _, on = pl.layout()
        assert nb <= most and sum(on) == len(gates)
    # a diagonal gate may not pass a non-diagonal one: H(0) . RZ(0) . H(0) keeps its order
    n = 12
    gates = [("H", (0,), ()), ("RZ", (0,), (0.7,)), ("H", (0,), ()), ("CZ", (0, 1), ()), ("RX", (1,), (0.3,)),
             ("CZ", (1, 2), ()), ("H", (2,), ()), ("CZ", (0, 2), ())]
    psi0 = inputs.random_state(n, 4)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        blocks = pl.tc_blocks()
    assert np.max(np.abs(run_blocks(n, blocks, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


@pytest.mark.parametrize("seed", [31, 32, 33, 34])
def test_fusion_with_many_diagonal_gates_reproduces_oracle(seed):
    # mostly diagonal gates on random qubits (so blocks split and diagonal
    # gates pass skipped ones), with non-diagonal gates in between
    n = 13
    names = ["RZ", "CZ", "RZZ", "T", "P", "S", "RX", "H", "CX"]
    gates = inputs.random_circuit(n, 240, seed, names=names, two_qubit_frac=0.5)
    psi0 = inputs.random_state(n, seed)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        blocks = pl.tc_blocks()
        pl.verify()
        _, _, on = pl.layout()
    assert sum(on) == len(gates) and len(blocks) > 3
    assert np.max(np.abs(run_blocks(n, blocks, psi0) - oracle.sv_run(n, gates, psi0))) <= 1e-12


def test_tfim_n34_plan_geometry_verifies():
    # the benchmark's n = 34 chain: every block's tile geometry checked on the host (operand
    # slots, coalescing, and for blocks without qubits 0..3 the direct write-back mapping:
    # thread t owns column t, loop step i chunk i)
    n = 34
    gates, _ = inputs.large_sv_tfim(n, 10)
    with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
        pl.verify()
        assert len(pl.tc_blocks()) == pl.info()["sweeps"]


@pytest.mark.parametrize("n", [12, 17, 26, 34])
def test_random_block_positions_verify(n):
    # one fused block per circuit, on five random qubits (blocks with and without qubits 0..3,
    # so both thread-role layouts): the host check of operand slots, coalescing and, for the
    # direct write-back layout, the thread-to-column mapping
    rng = np.random.default_rng(900 + n)
    for _ in range(12):
        qs = sorted(int(q) for q in rng.choice(n, size=5, replace=False))
        gates = [inputs.gate("CX", (qs[i], qs[i + 1])) for i in range(4)]
        gates += [inputs.gate("RY", (q,), (float(rng.uniform(-3, 3)),)) for q in qs]
        with sim.Plan(L.SV, n, gates, dtype=L.F32, flags=L.PLAN_TC) as pl:
            pl.verify()
            assert [sorted(b[0]) for b in pl.tc_blocks()] == [qs]
