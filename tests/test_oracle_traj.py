"""Pins of the oracle's quantum-trajectory unravelling (noisy state vectors,
the Monte-Carlo alternative to DM-Sim): reduction to the state-vector oracle
without noise, the trajectory average against the Kraus-form density matrix,
and closed forms of single jumps."""
import numpy as np

import oracle
from paper_2401_06861_gb300 import inputs
from tests import dense


def strong_noise(n, seed):
    return inputs.noise_params(n, seed=seed, p1=0.05, p2=0.1, t1q_ns=3000.0, t2q_ns=8000.0)


def test_without_noise_it_is_the_state_vector_run():
    n = 4
    g = inputs.random_circuit(n, 40, 11)
    assert oracle.traj_draws(g, None) == 0
    np.testing.assert_allclose(oracle.traj_run(n, g, None, []), oracle.sv_run(n, g), atol=1e-14)


def test_trajectory_average_is_the_kraus_density_matrix():
    n, M = 3, 3000
    g = inputs.random_circuit(n, 30, 12)
    noise = strong_noise(n, 13)
    d = oracle.traj_draws(g, noise)
    u = np.random.default_rng(14).random((M, d))
    psis = np.array([oracle.traj_run(n, g, noise, u[m]) for m in range(M)])
    outer = psis[:, :, None] * psis[:, None, :].conj()
    est, sd = outer.mean(axis=0), outer.std(axis=0) / np.sqrt(M)
    ref = oracle.dm_run(n, g, noise)
    assert np.all(np.abs(est - ref) <= 5 * sd + 1e-12)
    # noise really acts: the noisy state is far from the noiseless one
    psi0 = oracle.sv_run(n, g)
    assert np.abs(ref - np.outer(psi0, psi0.conj())).max() > 20 * sd.max()
    zt = inputs.z_terms(n)
    zest = np.mean([oracle.sv_expect(p, n, zt) for p in psis], axis=0)
    assert np.all(np.abs(zest - oracle.dm_expect(ref, n, zt)) <= 5 / np.sqrt(M))


def test_amplitude_damping_jump_closed_form():
    T1 = 100.0
    noise = dict(T1_us=np.array([T1]), T2_us=np.array([2 * T1]), t1q_ns=5000.0, t2q_ns=0.0, p1=0.0, p2=0.0,
                 readout_e=0.0)
    gamma = 1.0 - np.exp(-5000.0 / (T1 * 1e3))
    g = [inputs.gate("X", (0,))]
    assert oracle.traj_draws(g, noise) == 2
    # |1>: the decay happens exactly when the draw is below gamma
    np.testing.assert_allclose(oracle.traj_run(1, g, noise, [gamma * (1 - 1e-9), 0.5]), [1, 0], atol=1e-15)
    np.testing.assert_allclose(oracle.traj_run(1, g, noise, [gamma * (1 + 1e-9), 0.5]), [0, 1], atol=1e-15)
    # |+> without a jump: (1, sqrt(1 - gamma)) / norm; with T2 = 2 T1 there is no extra dephasing
    psi = oracle.traj_run(1, [inputs.gate("H", (0,))], noise, [0.999999, 0.999999])
    want = np.array([1.0, np.sqrt(1.0 - gamma)]) / np.sqrt(2.0 - gamma)
    np.testing.assert_allclose(psi, want, atol=1e-15)


def test_depolarising_draw_selects_the_pauli_string():
    P = [dense.I2, dense.X, dense.Y, dense.Z]
    p = 0.3
    noise1 = dict(T1_us=np.array([1.0]), T2_us=np.array([1.0]), t1q_ns=0.0, t2q_ns=0.0, p1=p, p2=0.0,
                  readout_e=0.0)
    g = [inputs.gate("H", (0,))]
    h = dense.one_qubit("H") @ np.array([1, 0])
    for s in (1, 2, 3):
        got = oracle.traj_run(1, g, noise1, [(s - 0.5) * p / 4])
        np.testing.assert_allclose(got, P[s] @ h, atol=1e-15)
    np.testing.assert_allclose(oracle.traj_run(1, g, noise1, [3 * p / 4 + 1e-9]), h, atol=1e-15)
    # two qubits: string s = a + 4 b puts Pauli a on q0 and b on q1
    p2 = 0.6
    noise2 = dict(T1_us=np.ones(2), T2_us=np.ones(2), t1q_ns=0.0, t2q_ns=0.0, p1=0.0, p2=p2, readout_e=0.0)
    g2 = [inputs.gate("H", (0,)), inputs.gate("CX", (0, 1))]
    base = dense.circuit_dense(2, g2) @ np.array([1, 0, 0, 0])
    for s in (1, 6, 11, 15):
        a, b = s & 3, s >> 2
        got = oracle.traj_run(2, g2, noise2, [(s - 0.5) * p2 / 16])
        want = dense.embed1(2, 1, P[b]) @ dense.embed1(2, 0, P[a]) @ base
        np.testing.assert_allclose(got, want, atol=1e-15)


def test_draw_margins_measure_the_distance_to_the_outcome_boundary():
    # amplitude damping from |1>: P1 = 1, the boundary is gamma itself; the
    # phase-damping draw of T2 = 2 T1 has rate 0 (no boundary: +inf)
    T1 = 100.0
    noise = dict(T1_us=np.array([T1]), T2_us=np.array([2 * T1]), t1q_ns=5000.0, t2q_ns=0.0, p1=0.0, p2=0.0,
                 readout_e=0.0)
    gamma = 1.0 - np.exp(-5000.0 / (T1 * 1e3))
    _, mg, kd = oracle.traj_run(1, [inputs.gate("X", (0,))], noise, [gamma * (1 - 1e-9), 0.5], margins=True)
    assert list(kd) == [1, 2]
    assert abs(mg[0] - 1e-9) <= 1e-15 and np.isinf(mg[1])
    # |+>: P1 = 1/2, the boundary is gamma / 2
    _, mg, _ = oracle.traj_run(1, [inputs.gate("H", (0,))], noise, [0.75 * gamma, 0.5], margins=True)
    assert abs(mg[0] - 0.5) <= 1e-12
    # depolarising: the draw's distance to the nearest of the sub-interval ends p/4, 2p/4, 3p/4, in units of p/4
    p = 0.3
    noise1 = dict(T1_us=np.array([1.0]), T2_us=np.array([1.0]), t1q_ns=0.0, t2q_ns=0.0, p1=p, p2=0.0,
                  readout_e=0.0)
    for x, want in ((0.5 * p / 4, 0.5), (1.9 * p / 4, 0.1), (3.2 * p / 4, 0.2), (0.9, 0.9 * 4 / p - 3)):
        _, mg, kd = oracle.traj_run(1, [inputs.gate("H", (0,))], noise1, [x], margins=True)
        assert list(kd) == [0] and abs(mg[0] - want) <= 1e-12, (x, mg, want)
