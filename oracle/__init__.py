"""CPU oracle: plain FP64 reference simulator (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this package.  The CUDA product path never imports it.

The arithmetic lives in ``nwq_oracle.c`` (plain C, FP64, gate by gate,
density matrices in Kraus form); this module only marshals numpy arrays.
It shares no code with the CUDA library: its gate-kind numbering, matrices
and channels are its own.

Parity pins (tests/test_oracle_*.py, marker "not gpu") tie every function
here to something other than itself: dense unitaries built from matrix
exponentials of Pauli generators, closed forms (Rabi oscillation, global
phase, depolarising and relaxation decay laws), exact diagonalisation and
the invariants of density matrices.

``tfim_fermion`` (numpy) gives exact expectation values of the Trotterised
Ising chain at any size through free fermions; it is pinned to this
package's state-vector oracle on small chains.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nwq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KIND = {"ID": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8,
        "SX": 9, "RX": 10, "RY": 11, "RZ": 12, "P": 13, "U3": 14, "MAT1": 15,
        "CX": 32, "CZ": 33, "SWAP": 34, "RZZ": 35, "MAT2": 36}


def build(force=False):
    """Compile the oracle with gcc (OpenMP for the density-matrix loops)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        Ip = ctypes.POINTER(ctypes.c_int)
        U64 = ctypes.POINTER(ctypes.c_uint64)
        c_int, c_dbl = ctypes.c_int, ctypes.c_double
        _lib.oracle_gate_matrix.argtypes = [c_int, D, D, D]
        _lib.oracle_sv_apply.argtypes = [D, c_int, c_int, Ip, D]
        _lib.oracle_sv_run.argtypes = [D, c_int, c_int, Ip, Ip, D, D]
        _lib.oracle_dm_run.argtypes = [D, c_int, c_int, Ip, Ip, D, D, c_int, D, D,
                                       c_dbl, c_dbl, c_dbl, c_dbl, ctypes.c_uint]
        _lib.oracle_dm_relax_direct.argtypes = [D, c_int, c_int, c_dbl, c_dbl, c_dbl]
        _lib.oracle_dm_relax_kraus.argtypes = [D, c_int, c_int, c_dbl, c_dbl, c_dbl]
        _lib.oracle_dm_depolarize.argtypes = [D, c_int, c_int, Ip, c_dbl]
        _lib.oracle_dm_unitary.argtypes = [D, c_int, c_int, Ip, D]
        _lib.oracle_sv_expect.argtypes = [D, c_int, c_int, U64, U64, D]
        _lib.oracle_dm_expect.argtypes = [D, c_int, c_int, U64, U64, D]
        _lib.oracle_sv_probs.argtypes = [D, c_int, c_dbl, D]
        _lib.oracle_dm_probs.argtypes = [D, c_int, c_dbl, D]
        _lib.oracle_traj_run.argtypes = [D, c_int, c_int, Ip, Ip, D, D, c_int, D, D, c_dbl, c_dbl, c_dbl, c_dbl,
                                         ctypes.c_uint, D, c_int, D, Ip]
        _lib.oracle_set_threads.argtypes = [c_int]
        _lib.oracle_max_threads.restype = c_int
        _lib.oracle_traj_draws.argtypes = [c_int, Ip, c_int, c_dbl, c_dbl, c_dbl, c_dbl, ctypes.c_uint]
    return _lib


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _encode(gates):
    ng = len(gates)
    kinds = np.zeros(max(ng, 1), np.int32)
    qs = np.zeros(2 * max(ng, 1), np.int32)
    th = np.zeros(3 * max(ng, 1), np.float64)
    mats = np.zeros(32 * max(ng, 1), np.float64)
    for g, (name, q, prm) in enumerate(gates):
        kinds[g] = KIND[name]
        qs[2 * g:2 * g + len(q)] = q
        if name.startswith("MAT"):
            m = np.asarray(prm, np.complex128).reshape(-1)
            mats[32 * g:32 * g + 2 * m.size] = np.stack([m.real, m.imag], -1).reshape(-1)
        else:
            th[3 * g:3 * g + len(prm)] = prm
    return ng, kinds, qs, th, mats


def gate_matrix(name, params=()):
    """The oracle's matrix of one gate (2x2 or 4x4 complex128)."""
    _, kinds, _, th, mats = _encode([(name, (0, 1) if KIND[name] >= 32 else (0,), params)])
    out = np.zeros(32, np.float64)
    nq = lib().oracle_gate_matrix(int(kinds[0]), _p(th), _p(mats), _p(out))
    d = 1 << nq
    return (out[0:2 * d * d:2] + 1j * out[1:2 * d * d:2]).reshape(d, d)


def zero_state(n):
    psi = np.zeros(1 << n, np.complex128)
    psi[0] = 1.0
    return psi


def sv_run(n, gates, psi0=None):
    """Apply ``gates`` gate by gate to psi0 (default |0..0>). Returns a new array."""
    psi = np.array(zero_state(n) if psi0 is None else psi0, dtype=np.complex128, copy=True)
    ng, kinds, qs, th, mats = _encode(gates)
    rc = lib().oracle_sv_run(_p(psi.view(np.float64)), n, ng, _p(kinds, ctypes.c_int),
                             _p(qs, ctypes.c_int), _p(th), _p(mats))
    if rc:
        raise ValueError("oracle_sv_run failed")
    return psi


def sv_run_inplace(psi, n, gates):
    """Apply ``gates`` to the complex128 array ``psi`` in place (no copy of the
    state; for timing large states)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << n
    ng, kinds, qs, th, mats = _encode(gates)
    rc = lib().oracle_sv_run(_p(psi.view(np.float64)), n, ng, _p(kinds, ctypes.c_int),
                             _p(qs, ctypes.c_int), _p(th), _p(mats))
    if rc:
        raise ValueError("oracle_sv_run failed")
    return psi


def set_threads(t):
    """OpenMP threads of the oracle's parallel loops."""
    lib().oracle_set_threads(int(t))


def max_threads():
    return int(lib().oracle_max_threads())


def dm_zero(n):
    N = 1 << n
    rho = np.zeros((N, N), np.complex128)
    rho[0, 0] = 1.0
    return rho


def dm_run(n, gates, noise=None, rho0=None):
    """Density-matrix run (row-major rho[r, c]); Kraus-form noise if ``noise``."""
    rho = np.array(dm_zero(n) if rho0 is None else rho0, dtype=np.complex128, copy=True, order="C")
    ng, kinds, qs, th, mats = _encode(gates)
    if noise is None:
        T1 = T2 = np.ones(max(n, 1))
        args = (0, T1, T2, 0.0, 0.0, 0.0, 0.0, 0)
    else:
        T1 = np.ascontiguousarray(noise["T1_us"], np.float64)
        T2 = np.ascontiguousarray(noise["T2_us"], np.float64)
        flags = (1 if noise.get("rz_virtual") else 0) | (2 if noise.get("depol_pauli_form") else 0)
        args = (1, T1, T2, noise["t1q_ns"], noise["t2q_ns"], noise["p1"], noise["p2"], flags)
    noisy, T1, T2, t1, t2, p1, p2, flags = args
    rc = lib().oracle_dm_run(_p(rho.view(np.float64)), n, ng, _p(kinds, ctypes.c_int),
                             _p(qs, ctypes.c_int), _p(th), _p(mats), noisy, _p(T1), _p(T2),
                             t1, t2, p1, p2, flags)
    if rc:
        raise ValueError(f"oracle_dm_run failed ({rc})")
    return rho


def _noise_args(n, noise):
    if noise is None:
        T1 = T2 = np.ones(max(n, 1))
        return (0, T1, T2, 0.0, 0.0, 0.0, 0.0, 0)
    T1 = np.ascontiguousarray(noise["T1_us"], np.float64)
    T2 = np.ascontiguousarray(noise["T2_us"], np.float64)
    flags = (1 if noise.get("rz_virtual") else 0) | (2 if noise.get("depol_pauli_form") else 0)
    return (1, T1, T2, noise["t1q_ns"], noise["t2q_ns"], noise["p1"], noise["p2"], flags)


def traj_draws(gates, noise):
    """Uniform draws one quantum trajectory of ``gates`` under ``noise`` consumes."""
    ng, kinds, qs, th, mats = _encode(gates)
    noisy, T1, T2, t1, t2, p1, p2, flags = _noise_args(1, noise)
    return int(lib().oracle_traj_draws(ng, _p(kinds, ctypes.c_int), noisy, ctypes.c_double(t1), ctypes.c_double(t2),
                                       ctypes.c_double(p1), ctypes.c_double(p2), flags))


def traj_run(n, gates, noise, uniforms, margins=False):
    """One quantum trajectory (final normalised state) driven by ``uniforms``.

    With ``margins``, returns (psi, margin, kind): per draw consumed, its
    relative distance to the nearest outcome boundary and its kind (0
    depolarising, 1 amplitude damping, 2 phase damping)."""
    psi = np.array(zero_state(n), dtype=np.complex128, copy=True)
    ng, kinds, qs, th, mats = _encode(gates)
    noisy, T1, T2, t1, t2, p1, p2, flags = _noise_args(n, noise)
    u = np.ascontiguousarray(uniforms, np.float64)
    mg = np.full(max(len(u), 1), np.inf)
    kd = np.full(max(len(u), 1), -1, np.int32)
    rc = lib().oracle_traj_run(_p(psi.view(np.float64)), n, ng, _p(kinds, ctypes.c_int), _p(qs, ctypes.c_int),
                               _p(th), _p(mats), noisy, _p(T1), _p(T2), ctypes.c_double(t1), ctypes.c_double(t2),
                               ctypes.c_double(p1), ctypes.c_double(p2), flags, _p(u), len(u),
                               _p(mg) if margins else None, _p(kd, ctypes.c_int) if margins else None)
    if rc < 0:
        raise ValueError(f"oracle_traj_run failed ({rc})")
    return (psi, mg[:rc], kd[:rc]) if margins else psi


def dm_depolarize(rho, n, qubits, p):
    rho = np.array(rho, np.complex128, copy=True, order="C")
    q = np.asarray(qubits, np.int32)
    lib().oracle_dm_depolarize(_p(rho.view(np.float64)), n, len(q), _p(q, ctypes.c_int), p)
    return rho


def dm_relax(rho, n, q, t_ns, T1_us, T2_us, direct=False):
    rho = np.array(rho, np.complex128, copy=True, order="C")
    if direct:
        lib().oracle_dm_relax_direct(_p(rho.view(np.float64)), n, q, t_ns, T1_us, T2_us)
    elif lib().oracle_dm_relax_kraus(_p(rho.view(np.float64)), n, q, t_ns, T1_us, T2_us):
        raise ValueError("T2 > 2 T1: no amplitude+phase damping Kraus split")
    return rho


def dm_unitary(rho, n, qubits, U):
    rho = np.array(rho, np.complex128, copy=True, order="C")
    q = np.asarray(qubits, np.int32)
    Ur = np.ascontiguousarray(np.asarray(U, np.complex128)).view(np.float64).reshape(-1).copy()
    lib().oracle_dm_unitary(_p(rho.view(np.float64)), n, len(q), _p(q, ctypes.c_int), _p(Ur))
    return rho


def _terms(terms):
    xm = np.array([t[0] for t in terms], np.uint64)
    zm = np.array([t[1] for t in terms], np.uint64)
    c = np.array([t[2] for t in terms], np.float64)
    return xm, zm, c


def sv_expect(psi, n, terms):
    """Per-term <psi|P|psi> (coefficients not applied)."""
    psi = np.ascontiguousarray(psi, np.complex128)
    xm, zm, _ = _terms(terms)
    out = np.zeros(len(terms))
    lib().oracle_sv_expect(_p(psi.view(np.float64)), n, len(terms), _p(xm, ctypes.c_uint64),
                           _p(zm, ctypes.c_uint64), _p(out))
    return out


def dm_expect(rho, n, terms):
    """Per-term Tr(rho P) (coefficients not applied)."""
    rho = np.ascontiguousarray(rho, np.complex128)
    xm, zm, _ = _terms(terms)
    out = np.zeros(len(terms))
    lib().oracle_dm_expect(_p(rho.view(np.float64)), n, len(terms), _p(xm, ctypes.c_uint64),
                           _p(zm, ctypes.c_uint64), _p(out))
    return out


def energy(values, terms):
    """sum_k coeff_k <P_k> from per-term values."""
    return float(sum(v * t[2] for v, t in zip(values, terms)))


def sv_probs(psi, n, readout_e=0.0):
    psi = np.ascontiguousarray(psi, np.complex128)
    out = np.zeros(1 << n)
    lib().oracle_sv_probs(_p(psi.view(np.float64)), n, readout_e, _p(out))
    return out


def dm_probs(rho, n, readout_e=0.0):
    rho = np.ascontiguousarray(rho, np.complex128)
    out = np.zeros(1 << n)
    lib().oracle_dm_probs(_p(rho.view(np.float64)), n, readout_e, _p(out))
    return out


def dm_to_vec(rho):
    """Row-major rho[r, c] -> column-stacked vec(rho)[r + N c]."""
    return np.ascontiguousarray(np.asarray(rho).T).reshape(-1)


def vec_to_dm(v, n):
    N = 1 << n
    return np.asarray(v).reshape(N, N).T.copy()
