"""OpenQASM 2.0 front end (host only): expressions, registers and
broadcasting, user gate definitions, controlled gates, round trip through the
writer, and rejected statements.  The programs are small hand-written ones."""
import math

import numpy as np
import pytest

from paper_2401_06861_gb300 import inputs, qasm
from tests import dense


@pytest.mark.parametrize("expr,val", [("pi/2", math.pi / 2), ("-pi/4+1", 1 - math.pi / 4), ("2^3^2", 2.0 ** 9),
                                      ("sin(pi/2)", 1.0), ("sqrt(2)*cos(0)", math.sqrt(2)), ("1e-3", 1e-3),
                                      (".5", 0.5), ("-(1+2)*3", -9.0), ("ln(exp(2))", 2.0), ("3/4/2", 0.375)])
def test_expressions(expr, val):
    assert qasm.evaluate(expr) == pytest.approx(val, abs=1e-15)


def test_registers_broadcast_user_gates_and_measure():
    prog = """
    OPENQASM 2.0;
    include "qelib1.inc";
    qreg a[2];
    qreg b[2];   // b[0] is qubit 2
    creg c[4];
    gate rot(th, ph) x, y { rz(th) x; cx x, y; ry(ph/2) y; }
    h a;
    cx a, b;
    rot(pi/3, -0.4) b[1], a[0];
    barrier a, b;
    u2(0.1, 0.2) b[0];
    measure a[1] -> c[1];
    """
    r = qasm.parse(prog)
    assert r["n"] == 4 and r["measured"] == [1]
    names = [g[0] for g in r["gates"]]
    assert names == ["H", "H", "CX", "CX", "RZ", "CX", "RY", "U3"]
    assert [g[1] for g in r["gates"]] == [(0,), (1,), (0, 2), (1, 3), (3,), (3, 0), (0,), (2,)]
    want = [inputs.gate("H", (0,)), inputs.gate("H", (1,)), inputs.gate("CX", (0, 2)), inputs.gate("CX", (1, 3)),
            inputs.gate("RZ", (3,), (math.pi / 3,)), inputs.gate("CX", (3, 0)), inputs.gate("RY", (0,), (-0.2,)),
            inputs.gate("U3", (2,), (math.pi / 2, 0.1, 0.2))]
    np.testing.assert_allclose(dense.circuit_dense(4, r["gates"]), dense.circuit_dense(4, want), atol=1e-14)


@pytest.mark.parametrize("name,params,U", [
    ("cp", (0.7,), np.diag([1, np.exp(0.7j)])), ("cu1", (-1.1,), np.diag([1, np.exp(-1.1j)])),
    ("crz", (0.5,), np.diag([np.exp(-0.25j), np.exp(0.25j)])), ("cy", (), dense.Y),
    ("ch", (), dense.one_qubit("H"))])
def test_controlled_gates(name, params, U):
    p = "(" + ",".join(map(str, params)) + ")" if params else ""
    r = qasm.parse(f"OPENQASM 2.0;\nqreg q[3];\n{name}{p} q[2], q[0];\n")
    got = dense.circuit_dense(3, r["gates"])
    # controlled-U with control q2, target q0: |c><c| (x) U on the target when c = 1
    P0 = dense.embed1(3, 2, np.diag([1, 0])) + 0j
    P1 = dense.embed1(3, 2, np.diag([0, 1])) + 0j
    want = P0 + P1 @ dense.embed1(3, 0, U)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_round_trip_through_the_writer():
    names = [g for g in inputs.GATE_NAMES if not g.startswith("MAT")]
    g = inputs.random_circuit(6, 200, 90, names=names)
    r = qasm.parse(qasm.dumps(6, g))
    assert r["n"] == 6 and len(r["gates"]) == len(g)
    for (a, qa, pa), (b, qb, pb) in zip(g, r["gates"]):
        assert a == b and qa == qb and np.allclose(pa, pb, rtol=0, atol=0)


@pytest.mark.parametrize("prog,msg", [
    ("OPENQASM 2.0; qreg q[1]; reset q[0];", "reset"), ("OPENQASM 2.0; qreg q[1]; creg c[1]; if(c==1) x q[0];", "if"),
    ("OPENQASM 2.0; qreg q[1]; foo q[0];", "unknown gate"), ("OPENQASM 2.0; qreg q[2]; cx q[0];", "count"),
    ("OPENQASM 2.0; qreg q[3]; ccx q[0], q[1], q[2];", "unknown gate"),
    ("OPENQASM 2.0; qreg q[2]; h q[2];", "out of range"), ("OPENQASM 3.0; qreg q[1];", "2.0"),
    ("OPENQASM 2.0; qreg q[2]; cx q[1], q[1];", "repeated"), ("OPENQASM 2.0; qreg q[1]; rx(pi/) q[0];", "expression"),
    ("OPENQASM 2.0; qreg a[2]; qreg b[3]; cx a, b;", "sizes"), ("OPENQASM 2.0;", "qreg")])
def test_rejected_programs(prog, msg):
    with pytest.raises(qasm.QasmError) as ei:
        qasm.parse(prog)
    assert msg in str(ei.value)
