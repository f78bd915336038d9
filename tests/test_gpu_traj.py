"""Quantum trajectories (noisy state vectors) on the GPU: per-trajectory
parity with the oracle on the same draws, and the trajectory average against
the density-matrix path."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim
from paper_2401_06861_gb300.sim import State

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


def strong_noise(n, seed):
    return inputs.noise_params(n, seed=seed, p1=0.05, p2=0.1, t1q_ns=3000.0, t2q_ns=8000.0)


def circuit(n, seed):
    names = [g for g in inputs.GATE_NAMES if not g.startswith("MAT")]
    return inputs.random_circuit(n, 60, seed, names=names)


@pytest.mark.parametrize("dtype", [L.F64, "f64_pipe", L.F32])
@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_each_trajectory_matches_the_oracle(n, dtype, monkeypatch):
    # F64 trajectories run in double words by default; NWQ_DW=0 selects the FP64 pipe
    if dtype == "f64_pipe":
        monkeypatch.setenv("NWQ_DW", "0")
        dtype = L.F64
    g, noise = circuit(n, 60 + n), strong_noise(n, 61 + n)
    terms = inputs.tfim_terms(n) + inputs.z_terms(n) + [(1, 3, 1.0)] if n > 1 else inputs.z_terms(n)
    coeffs = np.eye(len(terms))  # one row per term: every <P_k>
    ntraj = 48
    d = sim.trajectory_draws(n, g, noise)
    assert d == oracle.traj_draws(g, noise) and d > 0
    u = np.random.default_rng(62 + n).random((ntraj, d))
    got = sim.trajectories(n, g, noise, terms, coeffs, ntraj, dtype, uniforms=u)
    ref, near = [], []
    for t in range(ntraj):
        psi, margin, kind = oracle.traj_run(n, g, noise, u[t], margins=True)
        ref.append(oracle.sv_expect(psi, n, terms))
        # A jump is taken when the draw is below rate * P1, with P1 summed
        # from the stored state.  FP32 storage puts a relative error of at
        # most a few 2^-24 per gate on P1 (these circuits have 60 gates, so
        # below 1e-5); a relaxation draw within 1e-4 (relative) of its
        # threshold may therefore take the other branch in FP32.  The
        # depolarising draws are compared with FP64 parameters on both sides.
        near.append(bool(np.any((kind > 0) & (margin <= 1e-4))))
    ref, near = np.array(ref), np.array(near)
    err = np.abs(got - ref).max(axis=1)
    if dtype == L.F64:
        assert err.max() <= 1e-12
    else:  # every trajectory with no draw near a threshold matches at the FP32 tolerance
        assert err[~near].max() <= 1e-5, (err, near)
        assert near.mean() <= 0.1, near


def test_average_converges_to_the_density_matrix():
    n, ntraj = 6, 4096
    g, noise = circuit(n, 70), strong_noise(n, 71)
    terms = inputs.tfim_terms(n) + inputs.z_terms(n)
    got = sim.trajectories(n, g, noise, terms, np.eye(len(terms)), ntraj, L.F64, seed=72)
    with State(L.DM, n, L.F64) as st:
        st.apply(g, noise=noise)
        dm = st.expect(terms)
    mean, se = got.mean(axis=0), got.std(axis=0) / np.sqrt(ntraj)
    assert np.all(np.abs(mean - dm) <= 5 * se + 1e-12), (mean - dm, se)
    noiseless = oracle.sv_expect(oracle.sv_run(n, g), n, terms)
    assert np.abs(dm - noiseless).max() > 20 * se.max()  # the noise is visible


def test_noise_free_trajectories_are_the_state_vector():
    n = 7
    g = circuit(n, 80)
    terms = inputs.tfim_terms(n)
    got = sim.trajectories(n, g, None, terms, [[t[2] for t in terms]], 3, L.F64)
    assert sim.trajectory_draws(n, g, None) == 0
    ref = oracle.energy(oracle.sv_expect(oracle.sv_run(n, g), n, terms), terms)
    assert np.abs(got[:, 0] - ref).max() <= 1e-12


def test_trajectory_validation():
    n = 3
    g = [inputs.gate("H", (0,))]
    bad_noise = inputs.noise_params(n)
    bad_noise["T2_us"] = 3.0 * bad_noise["T1_us"]  # T2 > 2 T1: no amplitude-plus-phase damping split
    with pytest.raises(L.NwqError) as ei:
        sim.trajectories(n, g, bad_noise, inputs.z_terms(n), np.eye(n), 2)
    assert b"T2 <= 2 T1" in L.lib().nwq_last_error()
    with pytest.raises(L.NwqError):
        sim.trajectories(15, [inputs.gate("H", (0,))], None, inputs.z_terms(15), np.eye(15), 2)
