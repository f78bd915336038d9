"""Pins of the density-matrix oracle (Kraus form) against closed forms,
dense matrix algebra and the invariants of quantum channels."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import inputs
from tests import dense


def test_noiseless_dm_equals_dense_U_rho_Udag():
    n = 4
    gates = inputs.random_circuit(n, 40, 21)
    rho0 = inputs.random_density(n, 22)
    U = dense.circuit_dense(n, gates)
    np.testing.assert_allclose(oracle.dm_run(n, gates, None, rho0), U @ rho0 @ U.conj().T, atol=1e-13)


def test_noiseless_pure_state_matches_sv():
    n = 5
    gates = inputs.random_circuit(n, 50, 5)
    psi = dense.circuit_dense(n, gates)[:, 0]
    np.testing.assert_allclose(oracle.dm_run(n, gates), np.outer(psi, psi.conj()), atol=1e-13)


@pytest.mark.parametrize("qubits", [(1,), (0, 2), (2, 0)])
def test_depolarizing_equals_partial_trace_mix(qubits):
    n, p = 3, 0.13
    rho = inputs.random_density(n, 31)
    ref = (1 - p) * rho + p * dense.partial_trace_replace(rho, n, qubits)
    np.testing.assert_allclose(oracle.dm_depolarize(rho, n, qubits, p), ref, atol=1e-14)


def test_depolarizing_repeated_closed_form_and_fixed_point():
    n, p, k = 1, 0.05, 37
    rho = inputs.random_density(n, 3)
    r = rho
    for _ in range(k):
        r = oracle.dm_depolarize(r, n, (0,), p)
    ref = (1 - p) ** k * rho + (1 - (1 - p) ** k) * np.eye(2) / 2
    np.testing.assert_allclose(r, ref, atol=1e-14)
    full = oracle.dm_depolarize(rho, n, (0,), 1.0)
    np.testing.assert_allclose(full, np.eye(2) / 2, atol=1e-15)


def test_two_qubit_full_depolarizing_gives_maximally_mixed():
    n = 2
    rho = inputs.random_density(n, 8)
    np.testing.assert_allclose(oracle.dm_depolarize(rho, n, (0, 1), 1.0), np.eye(4) / 4, atol=1e-15)


def test_relaxation_decay_laws():
    T1, T2, t = 80.0, 60.0, 35.0  # us, us, ns
    rho = inputs.random_density(1, 17)
    out = oracle.dm_relax(rho, 1, 0, t, T1, T2)
    np.testing.assert_allclose(out[1, 1], rho[1, 1] * np.exp(-t / (T1 * 1e3)), atol=1e-15)
    np.testing.assert_allclose(abs(out[0, 1]), abs(rho[0, 1]) * np.exp(-t / (T2 * 1e3)), atol=1e-15)
    np.testing.assert_allclose(np.trace(out), 1.0, atol=1e-15)


def test_relaxation_kraus_matches_direct_action_and_converges_to_ground():
    n = 3
    rho = inputs.random_density(n, 19)
    for q, (T1, T2) in enumerate([(50.0, 30.0), (150.0, 120.0), (70.0, 140.0)]):
        a = oracle.dm_relax(rho, n, q, 300.0, T1, T2)
        b = oracle.dm_relax(rho, n, q, 300.0, T1, T2, direct=True)
        np.testing.assert_allclose(a, b, atol=1e-15)
    r = inputs.random_density(1, 4)
    for _ in range(200):
        r = oracle.dm_relax(r, 1, 0, 1e5, 50.0, 40.0)
    np.testing.assert_allclose(r, np.diag([1.0, 0.0]), atol=1e-12)


def test_relaxation_rejects_t2_above_2t1_in_kraus_form():
    with pytest.raises(ValueError):
        oracle.dm_relax(inputs.random_density(1, 1), 1, 0, 300.0, 50.0, 120.0)


def test_noisy_tfim_invariants():
    n = 5
    gates, noise = inputs.dm_noisy_tfim(n, steps=4)
    rho = oracle.dm_run(n, gates, noise)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.abs(rho - rho.conj().T).max() < 1e-14
    ev = np.linalg.eigvalsh(rho)
    assert ev.min() > -1e-13
    purity = np.real(np.trace(rho @ rho))
    assert purity < 1 - 1e-4  # noise made the state mixed
    # noise shrinks |<Z>| relative to the noiseless run (paper Fig. 3 trend)
    psi = oracle.sv_run(n, gates)
    z_clean = oracle.sv_expect(psi, n, inputs.z_terms(n))
    z_noisy = oracle.dm_expect(rho, n, inputs.z_terms(n))
    assert np.all(np.abs(z_noisy) <= np.abs(z_clean) + 1e-12)


def test_noisy_step_equals_channel_composition_by_hand():
    # one CX and one RX with the noise order gate -> depolarising -> relaxation
    n = 2
    noise = inputs.noise_params(n, seed=5)
    gates = [inputs.gate("CX", (0, 1)), inputs.gate("RX", (1,), (0.7,))]
    rho = inputs.random_density(n, 6)
    r = dense.gate_dense(n, gates[0]) @ rho @ dense.gate_dense(n, gates[0]).conj().T
    r = (1 - noise["p2"]) * r + noise["p2"] * dense.partial_trace_replace(r, n, (0, 1))
    for q in (0, 1):
        r = oracle.dm_relax(r, n, q, noise["t2q_ns"], noise["T1_us"][q], noise["T2_us"][q], direct=True)
    U = dense.gate_dense(n, gates[1])
    r = U @ r @ U.conj().T
    r = (1 - noise["p1"]) * r + noise["p1"] * dense.partial_trace_replace(r, n, (1,))
    r = oracle.dm_relax(r, n, 1, noise["t1q_ns"], noise["T1_us"][1], noise["T2_us"][1], direct=True)
    np.testing.assert_allclose(oracle.dm_run(n, gates, noise, rho), r, atol=1e-14)


def test_rz_virtual_flag_skips_noise_on_rz_only():
    n = 2
    noise = inputs.noise_params(n, seed=5, rz_virtual=True)
    rho = inputs.random_density(n, 6)
    g = [inputs.gate("RZ", (1,), (0.3,))]
    U = dense.gate_dense(n, g[0])
    np.testing.assert_allclose(oracle.dm_run(n, g, noise, rho), U @ rho @ U.conj().T, atol=1e-15)


def test_depolarizing_pauli_form_conversion():
    # Pauli form: p/3 on each of X, Y, Z  ==  depolarising parameter 4p/3
    n, p = 1, 0.03
    rho = inputs.random_density(n, 2)
    noise = inputs.noise_params(1, seed=1, t1q_ns=0.0, p1=p, depol_pauli_form=True)
    out = oracle.dm_run(n, [inputs.gate("ID", (0,))], noise, rho)
    ref = (1 - p) * rho + (p / 3) * sum(P @ rho @ P for P in (dense.X, dense.Y, dense.Z))
    np.testing.assert_allclose(out, ref, atol=1e-15)


def test_readout_scales_z_by_one_minus_two_e():
    n, e = 4, 0.02
    rho = oracle.dm_run(n, *inputs.dm_noisy_tfim(n, steps=3))
    p0 = oracle.dm_probs(rho, n, 0.0)
    p = oracle.dm_probs(rho, n, e)
    assert abs(p.sum() - 1) < 1e-14
    b = np.arange(1 << n)
    for i in range(n):
        s = 1 - 2 * ((b >> i) & 1)
        assert abs((p * s).sum() - (1 - 2 * e) * (p0 * s).sum()) < 1e-14
    for i in range(n - 1):
        s = (1 - 2 * ((b >> i) & 1)) * (1 - 2 * ((b >> (i + 1)) & 1))
        assert abs((p * s).sum() - (1 - 2 * e) ** 2 * (p0 * s).sum()) < 1e-14
    # equals the Kronecker product of the 2x2 confusion matrices
    C = np.array([[1 - e, e], [e, 1 - e]])
    Cn = np.array([[1.0]])
    for _ in range(n):
        Cn = np.kron(Cn, C)
    np.testing.assert_allclose(p, Cn @ p0, atol=1e-15)


def test_sv_probs_readout_matches_kronecker_confusion():
    n, e = 5, 0.07
    psi = inputs.random_state(n, 12)
    C = np.array([[1 - e, e], [e, 1 - e]])
    Cn = np.array([[1.0]])
    for _ in range(n):
        Cn = np.kron(Cn, C)
    np.testing.assert_allclose(oracle.sv_probs(psi, n, e), Cn @ np.abs(psi) ** 2, atol=1e-15)
