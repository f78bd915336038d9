"""The VQE optimiser loop (COBYLA, paper Sec. III) on host energies: no GPU."""
import numpy as np

from paper_2401_06861_gb300 import vqe


def test_cobyla_reaches_the_minimum_of_a_separable_landscape():
    a = np.linspace(0.3, 2.1, 6)

    def energy(t):  # minimum -6 at t = a + pi
        return float(np.sum(np.cos(np.asarray(t) - a)))

    r = vqe.minimize(energy, 6, starts=4, maxiter=3000, tol=1e-9)
    assert r["success"]
    assert abs(r["energy"] + 6.0) < 1e-8
    assert r["nfev"] == len(r["history"])
    assert np.all(r["history"] >= -6.0 - 1e-12)
    assert np.allclose(np.cos(r["theta"] - a), -1.0, atol=1e-4)


def test_start_is_the_best_of_the_scored_points_and_seeded():
    calls = []

    def batch(c):
        calls.append(len(c))
        return np.sum(c, axis=1)  # smallest sum wins

    def energy(t):
        return float(np.sum(t))

    r1 = vqe.minimize(energy, 3, starts=32, batch_energy=batch, maxiter=5)
    r2 = vqe.minimize(energy, 3, starts=32, batch_energy=batch, maxiter=5)
    assert calls == [32, 32]  # one batched call scores all starts
    cand = np.random.default_rng(4096).uniform(0.0, 2.0 * np.pi, size=(32, 3))
    best = cand[np.argmin(cand.sum(axis=1))]
    assert np.allclose(r1["history"][0], best.sum())  # COBYLA's first evaluation is x0
    assert np.array_equal(r1["theta"], r2["theta"])


def test_explicit_start_is_used():
    x0 = np.array([0.1, 0.2])
    seen = []
    vqe.minimize(lambda t: seen.append(np.array(t)) or float(np.sum(t ** 2)), 2, x0=x0, maxiter=5)
    assert np.allclose(seen[0], x0)
