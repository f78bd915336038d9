"""Pins of the oracle's Pauli expectations and TFIM energies."""
import numpy as np
import pytest
from scipy.sparse.linalg import eigsh
from scipy import sparse

import oracle
from paper_2401_06861_gb300 import inputs
from tests import dense


def test_sv_expect_matches_dense_pauli_matrices():
    n = 5
    psi = inputs.random_state(n, 3)
    terms = inputs.random_pauli_terms(n, 40, 4)
    got = oracle.sv_expect(psi, n, terms)
    ref = [np.real(psi.conj() @ dense.pauli_dense(n, x, z) @ psi) for x, z, _ in terms]
    np.testing.assert_allclose(got, ref, atol=1e-14)


def test_dm_expect_matches_dense_trace():
    n = 4
    rho = inputs.random_density(n, 8)
    terms = inputs.random_pauli_terms(n, 40, 9)
    got = oracle.dm_expect(rho, n, terms)
    ref = [np.real(np.trace(rho @ dense.pauli_dense(n, x, z))) for x, z, _ in terms]
    np.testing.assert_allclose(got, ref, atol=1e-14)


def test_pauli_y_convention():
    # |+i> = (|0> + i|1>)/sqrt2 has <Y> = +1
    psi = np.array([1, 1j]) / np.sqrt(2)
    assert abs(oracle.sv_expect(psi, 1, [(1, 1, 1.0)])[0] - 1.0) < 1e-15


def _tfim_sparse(n, J, h):
    N = 1 << n
    b = np.arange(N)
    diag = np.zeros(N)
    for i in range(n - 1):
        diag += -J * (1 - 2 * ((b >> i) & 1)) * (1 - 2 * ((b >> (i + 1)) & 1))
    H = sparse.diags(diag).tocsr()
    for i in range(n):
        H = H + sparse.csr_matrix((-h * np.ones(N), (b ^ (1 << i), b)), shape=(N, N))
    return H


@pytest.mark.parametrize("h", [0.5, 1.0, 2.0])
def test_vqe_energies_respect_the_variational_bound(h):
    n, layers = 8, 4
    H = _tfim_sparse(n, 1.0, h)
    e0 = eigsh(H, k=1, which="SA")[0][0]
    terms = inputs.tfim_terms(n, 1.0, h)
    params = inputs.hea_params(n, layers, 6, seed=1)
    for p in params:
        g, _ = inputs.hea_ansatz(n, layers, p)
        psi = oracle.sv_run(n, g)
        e = oracle.energy(oracle.sv_expect(psi, n, terms), terms)
        assert e >= e0 - 1e-12
        assert abs(e - np.real(psi.conj() @ (H @ psi))) < 1e-12


def test_energy_is_linear_in_h():
    n = 6
    g, _ = inputs.hea_ansatz(n, 2, inputs.hea_params(n, 2, 1, seed=3)[0])
    psi = oracle.sv_run(n, g)
    e = [oracle.energy(oracle.sv_expect(psi, n, inputs.tfim_terms(n, 1.0, h)), inputs.tfim_terms(n, 1.0, h))
         for h in (0.5, 1.0, 2.0)]
    assert abs((e[2] - e[1]) - 2 * (e[1] - e[0])) < 1e-13
