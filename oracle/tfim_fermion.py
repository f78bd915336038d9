"""Exact TFIM expectation values through free fermions (TEST INFRASTRUCTURE ONLY).

Only the tests may use this module; the CUDA product path never imports it.

The Trotterised transverse-field Ising chain of Sec. 3 (the spin chain of
Fig. 3: ZZ couplings on an open chain, an X field per site) is a circuit of
RZZ(theta) = exp(-i theta/2 Z_i Z_{i+1}) and RX(theta) = exp(-i theta/2 X_i)
gates.  Under the Jordan-Wigner map with Majorana operators

    a_{2i}   = X_0 ... X_{i-1} Z_i,
    a_{2i+1} = X_0 ... X_{i-1} Y_i,

both generators are quadratic: X_i = i a_{2i} a_{2i+1} and
Z_i Z_{i+1} = i a_{2i+1} a_{2i+2}, and Z_0 = a_0 is linear.  A gate
exp(-i phi (i a_p a_q)) maps, in the Heisenberg picture,

    a_p -> cos(2 phi) a_p + sin(2 phi) a_q,   a_q -> cos(2 phi) a_q - sin(2 phi) a_p,

so the whole circuit U acts on the 2n Majoranas by one rotation R in SO(2n)
(U^dag a_p U = sum_k R_pk a_k, R = R_L ... R_1 for gates 1..L), and

    <i a_p a_q>(t) = (R G0 R^T)_pq,   <a_p>(t) = (R g0)_p,

where G0 and g0 are the initial state's two- and one-point functions.  For
|0...0>: G0[2i+1, 2i+2] = <Z_i Z_{i+1}> = 1 (and -1 transposed), all other
entries 0 (every other product a_p a_q carries an X or Y), g0 = e_0.  This
needs no Gaussian initial state: the evolved observables are quadratic (or
linear), so two-point functions suffice.  Cost O(L n) for any n, so it gives
exact <Z_i Z_{i+1}>, <X_i>, <Z_0> and <H> for the 33- and 34-qubit chains.

A CX(i, i+1) RZ_{i+1}(theta) CX(i, i+1) triple is exactly RZZ(theta) on (i, i+1)
(CX conjugation maps Z_{i+1} to Z_i Z_{i+1}) and is read as such.
"""
from __future__ import annotations

import numpy as np


def _pairs(n, gates):
    """(p, q, phi) of each quadratic gate exp(-i phi (i a_p a_q)), in circuit order."""
    out = []
    k = 0
    while k < len(gates):
        name, qs, prm = gates[k][0], tuple(gates[k][1]), gates[k][2]
        if name == "RX":
            q = qs[0]
            out.append((2 * q, 2 * q + 1, 0.5 * float(prm[0])))
            k += 1
        elif name == "RZZ" and abs(qs[0] - qs[1]) == 1:
            i = min(qs)
            out.append((2 * i + 1, 2 * i + 2, 0.5 * float(prm[0])))
            k += 1
        elif (name == "CX" and k + 2 < len(gates) and qs[1] == qs[0] + 1 and gates[k + 1][0] == "RZ"
              and tuple(gates[k + 1][1]) == (qs[1],) and gates[k + 2][0] == "CX" and tuple(gates[k + 2][1]) == qs):
            i = qs[0]
            out.append((2 * i + 1, 2 * i + 2, 0.5 * float(gates[k + 1][2][0])))
            k += 3
        else:
            raise ValueError(f"gate {k} ({name} on {qs}) is not a nearest-neighbour RZZ or an RX")
    for p, q, _ in out:
        if not (0 <= p < q < 2 * n):
            raise ValueError("qubit out of range")
    return out


def majorana_rotation(n, gates):
    """R in SO(2n) with U^dag a_p U = sum_k R[p, k] a_k for the circuit U."""
    R = np.eye(2 * n)
    for p, q, phi in _pairs(n, gates):  # R <- R_j R, gate j after all earlier ones
        c, s = np.cos(2 * phi), np.sin(2 * phi)
        rp, rq = R[p].copy(), R[q].copy()
        R[p] = c * rp + s * rq
        R[q] = c * rq - s * rp
    return R


def tfim_observables(n, gates):
    """Exact <Z_i Z_{i+1}> (n-1), <X_i> (n) and <Z_0> after ``gates`` on |0...0>."""
    R = majorana_rotation(n, gates)
    G0 = np.zeros((2 * n, 2 * n))
    for i in range(n - 1):
        G0[2 * i + 1, 2 * i + 2] = 1.0
        G0[2 * i + 2, 2 * i + 1] = -1.0
    G = R @ G0 @ R.T
    zz = np.array([G[2 * i + 1, 2 * i + 2] for i in range(n - 1)])
    x = np.array([G[2 * i, 2 * i + 1] for i in range(n)])
    return {"zz": zz, "x": x, "z0": float(R[0, 0])}
