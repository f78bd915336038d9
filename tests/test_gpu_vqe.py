"""VQE for the Ising chain through the CUDA library (paper Sec. III, Fig. 4):
energies against the oracle, the variational bound against exact
diagonalisation, and the COBYLA loop reaching the ground energy."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, vqe

from tests.dense import pauli_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


def ground_energy(n, J=1.0, h=1.0):
    H = sum(c * pauli_dense(n, x, z) for x, z, c in inputs.tfim_terms(n, J, h))
    return float(np.linalg.eigvalsh(H)[0])


def oracle_energy(n, layers, theta, noise=None, J=1.0, h=1.0):
    gates, _ = inputs.hea_ansatz(n, layers, theta)
    terms = inputs.tfim_terms(n, J, h)
    if noise is None:
        return oracle.energy(oracle.sv_expect(oracle.sv_run(n, gates), n, terms), terms)
    return oracle.energy(oracle.dm_expect(oracle.dm_run(n, gates, noise), n, terms), terms)


@pytest.mark.parametrize("n,layers", [(4, 2), (6, 3)])
def test_energies_match_the_oracle(n, layers):
    thetas = inputs.hea_params(n, layers, 5, seed=77)
    noise = inputs.noise_params(n, seed=78)
    ef = vqe.NoiseFreeEnergy(n, layers, dtype=L.F64)
    en = vqe.NoisyEnergy(n, layers, noise, dtype=L.F64)
    got = ef.batch(thetas)
    for t, e in zip(thetas, got):
        assert abs(e - oracle_energy(n, layers, t)) <= 1e-12
        assert abs(ef(t) - e) <= 1e-13
        assert abs(en(t) - oracle_energy(n, layers, t, noise)) <= 1e-12
    ef.close()
    en.close()


def test_cobyla_vqe_noise_free_and_noisy():
    n, layers = 4, 3
    e0 = ground_energy(n)
    ef = vqe.NoiseFreeEnergy(n, layers, dtype=L.F64)
    r = vqe.minimize(ef, ef.nparams, starts=64, batch_energy=ef.batch, maxiter=4000, tol=1e-8)
    print(f"noise-free VQE n={n}: E={r['energy']:.6f} exact {e0:.6f} nfev={r['nfev']}")
    assert np.all(r["history"] >= e0 - 1e-9)  # variational bound at every evaluation
    assert r["energy"] - e0 <= 0.02 * abs(e0)
    noise = inputs.noise_params(n, seed=2401)
    en = vqe.NoisyEnergy(n, layers, noise, dtype=L.F64)
    rn = vqe.minimize(en, en.nparams, x0=r["theta"], maxiter=300, tol=1e-6)
    print(f"noisy VQE n={n}: E={rn['energy']:.6f} (noise-free optimum {r['energy']:.6f})")
    assert np.all(rn["history"] >= e0 - 1e-9)  # Tr(rho H) >= E0 for every state
    assert rn["energy"] > r["energy"]  # the device noise raises the reachable energy
    assert abs(rn["energy"] - oracle_energy(n, layers, rn["theta"], noise)) <= 1e-12
    ef.close()
    en.close()
