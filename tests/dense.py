"""Dense-matrix definitions used to pin the oracle (tests only).

Every one-qubit gate is defined here from the matrix exponential of its
Pauli generator (scipy.linalg.expm) or from a defining identity, not from a
retyped closed form, so a sign, factor or index slip in the oracle's own
matrices shows up as a mismatch.
"""
import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)


def rot(P, th):
    return expm(-0.5j * th * P)


def one_qubit(name, prm=()):
    if name == "ID":
        return I2
    if name == "X":
        return X
    if name == "Y":
        return Y
    if name == "Z":
        return Z
    if name == "RX":
        return rot(X, prm[0])
    if name == "RY":
        return rot(Y, prm[0])
    if name == "RZ":
        return rot(Z, prm[0])
    if name == "P":  # phase gate = RZ up to the global phase e^{i l/2}
        return np.exp(0.5j * prm[0]) * rot(Z, prm[0])
    if name == "S":
        return np.exp(0.25j * np.pi) * rot(Z, np.pi / 2)
    if name == "SDG":
        return np.exp(-0.25j * np.pi) * rot(Z, -np.pi / 2)
    if name == "T":
        return np.exp(0.125j * np.pi) * rot(Z, np.pi / 4)
    if name == "TDG":
        return np.exp(-0.125j * np.pi) * rot(Z, -np.pi / 4)
    if name == "H":  # pi rotation about (x+z)/sqrt2, times i
        return 1j * rot((X + Z) / np.sqrt(2), np.pi)
    if name == "SX":  # sqrt(X) with eigenvalues 1, i: e^{i pi/4} RX(pi/2)
        return np.exp(0.25j * np.pi) * rot(X, np.pi / 2)
    if name == "U3":  # ZYZ Euler form with phase e^{i(p+l)/2}
        th, ph, la = prm
        return np.exp(0.5j * (ph + la)) * rot(Z, ph) @ rot(Y, th) @ rot(Z, la)
    if name == "MAT1":
        return np.asarray(prm, complex)
    raise KeyError(name)


def basis_op(n, fn):
    """Matrix of the linear map |b> -> fn(b) = list of (coef, b')."""
    N = 1 << n
    M = np.zeros((N, N), complex)
    for b in range(N):
        for c, bb in fn(b):
            M[bb, b] += c
    return M


def embed1(n, q, U):
    """U on qubit q of n (qubit q = bit q), via Kronecker products."""
    ops = [I2] * n
    ops[q] = U
    M = np.array([[1.0 + 0j]])
    for k in reversed(range(n)):  # most significant qubit first
        M = np.kron(M, ops[k])
    return M


def two_qubit_dense(n, name, q0, q1, prm=()):
    if name == "CX":
        return basis_op(n, lambda b: [(1.0, b ^ (1 << q1) if (b >> q0) & 1 else b)])
    if name == "CZ":
        return basis_op(n, lambda b: [(-1.0 if ((b >> q0) & 1) and ((b >> q1) & 1) else 1.0, b)])
    if name == "SWAP":
        def sw(b):
            b0, b1 = (b >> q0) & 1, (b >> q1) & 1
            bb = (b & ~((1 << q0) | (1 << q1))) | (b0 << q1) | (b1 << q0)
            return [(1.0, bb)]
        return basis_op(n, sw)
    if name == "RZZ":
        return expm(-0.5j * prm[0] * embed1(n, q0, Z) @ embed1(n, q1, Z))
    if name == "MAT2":
        M4 = np.asarray(prm, complex)

        def f(b):
            j = ((b >> q0) & 1) | (((b >> q1) & 1) << 1)
            base = b & ~((1 << q0) | (1 << q1))
            return [(M4[r, j], base | ((r & 1) << q0) | ((r >> 1) << q1)) for r in range(4)]
        return basis_op(n, f)
    raise KeyError(name)


def gate_dense(n, g):
    name, qs, prm = g
    if len(qs) == 1:
        return embed1(n, qs[0], one_qubit(name, prm))
    return two_qubit_dense(n, name, qs[0], qs[1], prm)


def circuit_dense(n, gates):
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        U = gate_dense(n, g) @ U
    return U


def pauli_dense(n, x, z):
    """i^{|x&z|} X^x Z^z as a dense matrix (built from single-qubit Paulis)."""
    M = np.eye(1 << n, dtype=complex)
    for q in range(n):
        xq, zq = (x >> q) & 1, (z >> q) & 1
        P = I2
        if xq and zq:
            P = Y
        elif xq:
            P = X
        elif zq:
            P = Z
        M = embed1(n, q, P) @ M
    return M


def partial_trace_replace(rho, n, qubits):
    """Tr_S(rho) (x) I_S / 2^|S| with the identity placed back on S."""
    N = 1 << n
    k = len(qubits)
    out = np.zeros_like(rho)
    for r in range(N):
        for c in range(N):
            mask = sum(1 << q for q in qubits)
            if (r & mask) != (c & mask):
                continue
            acc = 0
            for sub in range(1 << k):
                bits = sum(((sub >> j) & 1) << q for j, q in enumerate(qubits))
                acc += rho[(r & ~mask) | bits, (c & ~mask) | bits]
            out[r, c] = acc / (1 << k)
    return out


def apply_local(psi, n, qs, U):
    """psi <- U acting on qubits qs (local index bit t <-> qubit qs[t]), by index gathering."""
    others = [q for q in range(n) if q not in qs]
    r = np.arange(1 << (n - len(qs)))
    base = np.zeros_like(r)
    for i, q in enumerate(others):
        base |= ((r >> i) & 1) << q
    j = np.arange(1 << len(qs))
    off = np.zeros_like(j)
    for i, q in enumerate(qs):
        off |= ((j >> i) & 1) << q
    idx = base[:, None] | off[None, :]
    out = psi.copy()
    out[idx] = psi[idx] @ np.asarray(U).T
    return out
