"""Seeded synthetic inputs: circuits, noise parameters and Pauli terms.

This module only *describes* workloads.  It builds gate lists, noise
parameter arrays and Hamiltonian term lists; it applies no gate, channel
or reduction.  Both the CUDA path and the CPU oracle are fed from it, and
it imports neither.

Gate format: a tuple ``(name, qubits, params)``.
  name    one of GATE_NAMES
  qubits  tuple of ints (1 or 2 entries).  For two-qubit gates the first
          qubit is the low bit of the 2-qubit local index (control for CX).
  params  tuple of floats (angles, radians), or for MAT1/MAT2 a complex
          numpy array of shape (2, 2) / (4, 4) in the local basis
          j = b(q0) + 2 b(q1).

Qubit q is bit q of the amplitude index (little-endian).

Workloads follow the TFIM time-evolution and VQE use cases of the paper
(Sec. III: transverse-field Ising chain, device noise model with
depolarising, thermal-relaxation and measurement noise; VQE for the Ising
model).  The paper gives no numbers for them, so the sizes below are the
synthetic stand-ins named in each function.
"""
from __future__ import annotations

import numpy as np

ONE_QUBIT = ("ID", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "SX",
             "RX", "RY", "RZ", "P", "U3", "MAT1")
TWO_QUBIT = ("CX", "CZ", "SWAP", "RZZ", "MAT2")
GATE_NAMES = ONE_QUBIT + TWO_QUBIT
N_PARAMS = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "RZZ": 1, "U3": 3}


def gate(name, qubits, params=()):
    if name not in GATE_NAMES:
        raise ValueError(f"unknown gate {name}")
    return (name, tuple(int(q) for q in qubits), params if name.startswith("MAT") else tuple(float(p) for p in params))


# ---------------------------------------------------------------- TFIM
def tfim_trotter(n, J=1.0, h=1.0, dt=0.05, steps=40):
    """First-order Trotter circuit of the open transverse-field Ising chain.

    Per step: for each bond (i, i+1), ascending: CX(i,i+1), RZ_{i+1}(2 J dt),
    CX(i,i+1); then RX_i(2 h_i dt) on every qubit.  ``h`` is a scalar or a
    length-n array (per-qubit field).
    """
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    g = []
    for _ in range(steps):
        for i in range(n - 1):
            g.append(gate("CX", (i, i + 1)))
            g.append(gate("RZ", (i + 1,), (2.0 * J * dt,)))
            g.append(gate("CX", (i, i + 1)))
        for i in range(n):
            g.append(gate("RX", (i,), (2.0 * float(hs[i]) * dt,)))
    return g


def tfim_terms(n, J=1.0, h=1.0):
    """Pauli terms (x_mask, z_mask, coeff) of H = -J sum Z_i Z_{i+1} - sum h_i X_i."""
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    t = [(0, (1 << i) | (1 << (i + 1)), -float(J)) for i in range(n - 1)]
    t += [(1 << i, 0, -float(hs[i])) for i in range(n)]
    return t


def z_terms(n):
    """<Z_i> for every qubit, as unit-coefficient Pauli terms."""
    return [(0, 1 << i, 1.0) for i in range(n)]


def zz_terms(n):
    return [(0, (1 << i) | (1 << (i + 1)), 1.0) for i in range(n - 1)]


def x_terms(n):
    return [(1 << i, 0, 1.0) for i in range(n)]


# ---------------------------------------------------------------- VQE ansatz
def hea_ansatz(n, layers, params=None):
    """Hardware-efficient ansatz: per layer RY(q) then RZ(q) on every qubit,
    then a CX ladder CX(q, q+1), q ascending.  Parameter index of RY on
    qubit q in layer l is l*2n + 2q, of RZ l*2n + 2q + 1.

    Returns (gates, param_index) where param_index[k] is the parameter slot
    used by gate k (-1 for fixed gates).  If ``params`` is None the angles
    are left at 0 and only the slots matter.
    """
    g, idx = [], []
    for l in range(layers):
        for q in range(n):
            for r, name in ((0, "RY"), (1, "RZ")):
                k = l * 2 * n + 2 * q + r
                th = 0.0 if params is None else float(params[k])
                g.append(gate(name, (q,), (th,)))
                idx.append(k)
        for q in range(n - 1):
            g.append(gate("CX", (q, q + 1)))
            idx.append(-1)
    return g, idx


def hea_params(n, layers, nsets, seed=4096):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * np.pi, size=(nsets, layers * 2 * n))


# ---------------------------------------------------------------- noise
def noise_params(n, seed=2401, t1q_ns=35.0, t2q_ns=300.0, p1=1e-3, p2=1e-2,
                 readout_e=0.02, rz_virtual=False, depol_pauli_form=False):
    """Device noise model with seeded per-qubit T1/T2 (microseconds).

    T1 ~ U(50, 150) us, then T2 ~ U(30, min(2 T1, 120)) us, drawn in that
    order from numpy's default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    T1 = rng.uniform(50.0, 150.0, n)
    T2 = rng.uniform(30.0, np.minimum(2.0 * T1, 120.0))
    return dict(T1_us=T1, T2_us=T2, t1q_ns=float(t1q_ns), t2q_ns=float(t2q_ns),
                p1=float(p1), p2=float(p2), readout_e=float(readout_e),
                rz_virtual=bool(rz_virtual), depol_pauli_form=bool(depol_pauli_form))


# ---------------------------------------------------------------- random tests
def random_unitary(dim, rng):
    """Haar-ish random unitary via QR of a complex Gaussian matrix."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))


def random_circuit(n, ngates, seed, names=None, two_qubit_frac=0.35):
    """Random circuit over every gate kind (or ``names``), seeded."""
    rng = np.random.default_rng(seed)
    names = list(names or GATE_NAMES)
    ones = [g for g in names if g in ONE_QUBIT]
    twos = [g for g in names if g in TWO_QUBIT] if n >= 2 else []
    out = []
    for _ in range(ngates):
        if twos and (not ones or rng.random() < two_qubit_frac):
            name = twos[rng.integers(len(twos))]
            a, b = rng.choice(n, size=2, replace=False)
            qs = (int(a), int(b))
        else:
            name = ones[rng.integers(len(ones))]
            qs = (int(rng.integers(n)),)
        if name == "MAT1":
            p = random_unitary(2, rng)
        elif name == "MAT2":
            p = random_unitary(4, rng)
        else:
            p = tuple(rng.uniform(-np.pi, np.pi, N_PARAMS.get(name, 0)))
        out.append(gate(name, qs, p))
    return out


def random_state(n, seed):
    """Normalised random complex128 state vector of 2^n amplitudes."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def random_density(n, seed, rank=None):
    """Random mixed state rho = A A^dag / Tr, row-major (2^n, 2^n) complex128."""
    rng = np.random.default_rng(seed)
    N = 1 << n
    r = rank or N
    a = rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))
    rho = a @ a.conj().T
    return rho / np.trace(rho).real


def random_pauli_terms(n, nterms, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nterms):
        x = int(rng.integers(0, 1 << n))
        z = int(rng.integers(0, 1 << n))
        out.append((x, z, float(rng.uniform(-1, 1))))
    return out


# ---------------------------------------------------------------- workloads
def dm_noisy_tfim(n, steps=20, seed=2401):
    """Noisy TFIM workload: n-qubit chain, J = h = 1, dt = 0.05, ``steps``
    Trotter steps, the seeded device noise model above."""
    return tfim_trotter(n, 1.0, 1.0, 0.05, steps), noise_params(n, seed)


def large_sv_tfim(n, steps=10, seed=3334):
    """TFIM Trotter circuit with random per-qubit field h_i ~ U(0.5, 2)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.5, 2.0, n)
    return tfim_trotter(n, 1.0, h, 0.05, steps), h


# ---------------------------------------------------------------- serving stream
def serve_requests(rate=200.0, duration=60.0, seed=200, sv_frac=0.7, sv_n=(8, 26), dm_n=(6, 12),
                   trotter_steps=(5, 50), hea_layers=(2, 6)):
    """Poisson request stream for the serving loop.

    Each request is a dict: id, arrival (s), kind ("sv" or "dm"), n, family
    ("trotter" or "hea"), gates, noise (dm only), z_terms and h_terms (TFIM,
    J = h = 1).  Inter-arrival times are exponential with mean 1/rate; 70%
    state-vector requests with n ~ U{8..26}, 30% density-matrix requests with
    n ~ U{6..12}; half Trotter circuits (steps ~ U{5..50}), half hardware-
    efficient ansatz circuits (layers ~ U{2..6}, angles ~ U(0, 2 pi)); the DM
    requests carry the seeded device noise model of ``noise_params``.
    """
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        kind = "sv" if rng.random() < sv_frac else "dm"
        lo, hi = sv_n if kind == "sv" else dm_n
        n = int(rng.integers(lo, hi + 1))
        if rng.random() < 0.5:
            fam = "trotter"
            gates = tfim_trotter(n, 1.0, 1.0, 0.05, int(rng.integers(trotter_steps[0], trotter_steps[1] + 1)))
        else:
            fam = "hea"
            layers = int(rng.integers(hea_layers[0], hea_layers[1] + 1))
            gates, _ = hea_ansatz(n, layers, rng.uniform(0.0, 2.0 * np.pi, layers * 2 * n))
        req = dict(id=len(out), arrival=t, kind=kind, n=n, family=fam, gates=gates,
                   z_terms=z_terms(n), h_terms=tfim_terms(n))
        if kind == "dm":
            req["noise"] = noise_params(n, seed=int(rng.integers(1 << 30)))
        out.append(req)
    return out
