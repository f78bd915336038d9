"""Pins for the free-fermion TFIM oracle: it must agree, term by term, with the
gate-by-gate state-vector oracle (itself pinned to dense unitaries) on small
chains, for every field, coupling, time step and depth tried, and obey the
closed forms of its special cases."""
import numpy as np
import pytest

import oracle
from oracle import tfim_fermion as ff
from paper_2401_06861_gb300 import inputs


def _sv_values(n, gates):
    psi = oracle.sv_run(n, gates)
    zz = oracle.sv_expect(psi, n, inputs.zz_terms(n))
    x = oracle.sv_expect(psi, n, inputs.x_terms(n))
    z0 = oracle.sv_expect(psi, n, [(0, 1, 1.0)])[0]
    return np.real(zz), np.real(x), float(np.real(z0))


@pytest.mark.parametrize("n,J,steps,seed", [(2, 1.0, 7, 1), (3, 0.7, 12, 2), (5, 1.3, 9, 3), (8, -0.4, 6, 4),
                                            (10, 1.0, 10, 5)])
def test_free_fermion_matches_the_state_vector_oracle(n, J, steps, seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 2.0, n)
    dt = float(rng.uniform(0.02, 0.3))
    gates = inputs.tfim_trotter(n, J, h, dt, steps)
    got = ff.tfim_observables(n, gates)
    zz, x, z0 = _sv_values(n, gates)
    assert np.max(np.abs(got["zz"] - zz)) <= 1e-12
    assert np.max(np.abs(got["x"] - x)) <= 1e-12
    assert abs(got["z0"] - z0) <= 1e-12


def test_rzz_gates_and_mixed_order():
    # explicit RZZ gates, bonds in random order, fields interleaved
    n = 7
    rng = np.random.default_rng(11)
    gates = []
    for _ in range(60):
        if rng.random() < 0.5:
            i = int(rng.integers(n - 1))
            gates.append(inputs.gate("RZZ", (i + 1, i) if rng.random() < 0.5 else (i, i + 1),
                                     (float(rng.uniform(-3, 3)),)))
        else:
            gates.append(inputs.gate("RX", (int(rng.integers(n)),), (float(rng.uniform(-3, 3)),)))
    got = ff.tfim_observables(n, gates)
    zz, x, z0 = _sv_values(n, gates)
    assert np.max(np.abs(got["zz"] - zz)) <= 1e-12
    assert np.max(np.abs(got["x"] - x)) <= 1e-12
    assert abs(got["z0"] - z0) <= 1e-12


def test_closed_forms():
    n = 33
    rng = np.random.default_rng(3334)
    h = rng.uniform(0.5, 2.0, n)
    # J = 0: independent Rabi oscillations in the Y-Z plane: <X_i> = 0,
    # <Z_i Z_{i+1}> = cos(phi_i) cos(phi_{i+1}), <Z_0> = cos(phi_0)
    phi = 2 * h * 0.05 * 10
    r = ff.tfim_observables(n, inputs.tfim_trotter(n, 0.0, h, 0.05, 10))
    assert np.max(np.abs(r["x"])) <= 1e-13
    assert np.max(np.abs(r["zz"] - np.cos(phi[:-1]) * np.cos(phi[1:]))) <= 1e-13
    assert abs(r["z0"] - np.cos(phi[0])) <= 1e-13
    # h = 0: |0...0> is an eigenstate of every ZZ, nothing moves
    r = ff.tfim_observables(n, inputs.tfim_trotter(n, 1.0, 0.0, 0.05, 10))
    assert np.max(np.abs(r["zz"] - 1.0)) <= 1e-13 and np.max(np.abs(r["x"])) <= 1e-13 and r["z0"] == 1.0
    # the rotation stays orthogonal over a full-size circuit
    R = ff.majorana_rotation(n, inputs.large_sv_tfim(n, 10)[0])
    assert np.max(np.abs(R @ R.T - np.eye(2 * n))) <= 1e-12


def test_rejects_other_gates():
    with pytest.raises(ValueError):
        ff.tfim_observables(3, [inputs.gate("H", (0,))])
    with pytest.raises(ValueError):
        ff.tfim_observables(3, [inputs.gate("RZZ", (0, 2), (0.1,))])
