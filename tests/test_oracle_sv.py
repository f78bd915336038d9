"""Pins of the state-vector oracle against definitions other than itself."""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2401_06861_gb300 import inputs
from tests import dense


@pytest.mark.parametrize("name", inputs.ONE_QUBIT)
def test_one_qubit_matrices_match_generator_definitions(name):
    rng = np.random.default_rng(7)
    for _ in range(3):
        if name == "MAT1":
            prm = inputs.random_unitary(2, rng)
        else:
            prm = tuple(rng.uniform(-np.pi, np.pi, inputs.N_PARAMS.get(name, 0)))
        np.testing.assert_allclose(oracle.gate_matrix(name, prm), dense.one_qubit(name, prm), atol=1e-14)


@pytest.mark.parametrize("name", inputs.TWO_QUBIT)
def test_two_qubit_matrices_match_basis_action(name):
    rng = np.random.default_rng(11)
    prm = inputs.random_unitary(4, rng) if name == "MAT2" else tuple(rng.uniform(-3, 3, inputs.N_PARAMS.get(name, 0)))
    # on 2 qubits with q0 = bit 0 and q1 = bit 1 the local basis is the full basis
    np.testing.assert_allclose(oracle.gate_matrix(name, prm), dense.two_qubit_dense(2, name, 0, 1, prm), atol=1e-14)


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (5, 4), (6, 5)])
def test_random_circuits_match_dense_unitary(n, seed):
    gates = inputs.random_circuit(n, 60, seed)
    psi0 = inputs.random_state(n, seed + 100)
    U = dense.circuit_dense(n, gates)
    np.testing.assert_allclose(oracle.sv_run(n, gates, psi0), U @ psi0, atol=1e-13)


def test_reversed_qubit_pairs_are_distinct():
    # CX(0,2) and CX(2,0) differ; a transposed local basis would confuse them
    n = 3
    psi0 = inputs.random_state(n, 9)
    a = oracle.sv_run(n, [inputs.gate("CX", (0, 2))], psi0)
    b = oracle.sv_run(n, [inputs.gate("CX", (2, 0))], psi0)
    np.testing.assert_allclose(a, dense.two_qubit_dense(n, "CX", 0, 2) @ psi0, atol=1e-15)
    np.testing.assert_allclose(b, dense.two_qubit_dense(n, "CX", 2, 0) @ psi0, atol=1e-15)
    assert np.abs(a - b).max() > 1e-3


def _tfim_ops(n):
    zz = sum(dense.embed1(n, i, dense.Z) @ dense.embed1(n, i + 1, dense.Z) for i in range(n - 1))
    xs = sum(dense.embed1(n, i, dense.X) for i in range(n))
    return zz, xs


def test_tfim_n10_40_steps_matches_trotter_product_of_exponentials():
    # The literal gate list: per step exp(-i J dt sum ZZ) then exp(-i h dt sum X).
    n, J, h, dt, steps = 10, 1.0, 1.0, 0.05, 40
    zz, xs = _tfim_ops(n)
    U_step = expm(-1j * h * dt * xs) @ expm(-1j * J * dt * zz)
    ref = np.linalg.matrix_power(U_step, steps)[:, 0]
    psi = oracle.sv_run(n, inputs.tfim_trotter(n, J, h, dt, steps))
    assert np.abs(psi - ref).max() < 1e-12
    # ... and is within the first-order Trotter error of the exact evolution
    # under J sum ZZ + h sum X (the literal gate signs), whose Z expectations
    # coincide with those of e^{-iHt} for H = -J sum ZZ - h sum X.
    exact = expm(-1j * steps * dt * (J * zz + h * xs))[:, 0]
    assert np.abs(psi - exact).max() < 0.05
    exact_h = expm(-1j * steps * dt * (-J * zz - h * xs))[:, 0]
    np.testing.assert_allclose(np.conj(exact_h), exact, atol=1e-12)


def test_rabi_closed_form_when_J_is_zero():
    n, dt, steps = 7, 0.05, 13
    h = np.linspace(0.5, 2.0, n)
    psi = oracle.sv_run(n, inputs.tfim_trotter(n, 0.0, h, dt, steps))
    phi = 2 * h * dt * steps
    z = oracle.sv_expect(psi, n, inputs.z_terms(n))
    np.testing.assert_allclose(z, np.cos(phi), atol=1e-13)
    # product state: amplitude of b is prod_i (cos(phi_i/2) or -i sin(phi_i/2))
    b = np.arange(1 << n)
    amp = np.ones(1 << n, complex)
    for i in range(n):
        bit = (b >> i) & 1
        amp *= np.where(bit, -1j * np.sin(phi[i] / 2), np.cos(phi[i] / 2))
    np.testing.assert_allclose(psi, amp, atol=1e-13)


def test_global_phase_closed_form_when_h_is_zero():
    n, J, dt, steps = 6, 1.0, 0.05, 9
    psi = oracle.sv_run(n, inputs.tfim_trotter(n, J, 0.0, dt, steps))
    ref = np.zeros(1 << n, complex)
    ref[0] = np.exp(-1j * J * dt * (n - 1) * steps)
    np.testing.assert_allclose(psi, ref, atol=1e-14)


def test_norm_is_preserved():
    n = 8
    psi = oracle.sv_run(n, inputs.random_circuit(n, 200, 3), inputs.random_state(n, 4))
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_golden_tfim_n4_trajectory():
    """Fixture written by tests/golden/make_golden.py from the oracle; this
    guards against silent changes of the oracle's arithmetic."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "tfim_n4_z_trajectory.json")
    g = json.load(open(path))
    n = g["n"]
    psi = oracle.zero_state(n)
    step = inputs.tfim_trotter(n, g["J"], g["h"], g["dt"], 1)
    zz, xs = _tfim_ops(n)
    U_step = expm(-1j * g["h"] * g["dt"] * xs) @ expm(-1j * g["J"] * g["dt"] * zz)
    ref = np.eye(1 << n)[:, 0].astype(complex)
    for k, row in enumerate(g["z"]):
        psi = oracle.sv_run(n, step, psi)
        np.testing.assert_allclose(oracle.sv_expect(psi, n, inputs.z_terms(n)), row, atol=1e-14)
        ref = U_step @ ref
        zref = [np.real(ref.conj() @ dense.embed1(n, i, dense.Z) @ ref) for i in range(n)]
        np.testing.assert_allclose(row, zref, atol=1e-13)
