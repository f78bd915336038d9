"""ctypes binding of the C ABI declared in include/nwqgb.h.

Argument marshalling only: every step of the simulation runs in the CUDA
library ``libnwqgb.so``.  Loading fails loudly if the library is missing;
there is no CPU fallback.  Device memory and streams may come from PyTorch
(pass ``tensor.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import atexit
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnwqgb.so")

OK, EINVAL, ENOMEM, ECUDA, EBUDGET, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
F32, F64 = 1, 2
SV, DM = 1, 2
PLAN_FUSED, PLAN_PLAIN, PLAN_NO_MERGE, PLAN_NO_RESCALE, PLAN_INTERPRETED, PLAN_TC, PLAN_COMMUTE = 0, 1, 2, 4, 8, 16, 32
PLAN_DW, PLAN_FP64, PLAN_NO_COMMUTE = 64, 128, 256
PROBE_FP64_FMA, PROBE_FP32_FMA = 0, 1
EXPECT_TERMS, EXPECT_SUM, EXPECT_NORMALIZE = 0, 1, 2
NOISE_RZ_VIRTUAL, NOISE_DEPOL_PAULI_FORM = 1, 2
NOALLOC_MAX_TERMS = 256
BATCH_GRAPH = 1
BATCH_FP64_PIPE = 2

GATE_KIND = {"ID": 1, "X": 2, "Y": 3, "Z": 4, "H": 5, "S": 6, "SDG": 7, "T": 8, "TDG": 9, "SX": 10,
             "RX": 11, "RY": 12, "RZ": 13, "P": 14, "U3": 15, "MAT1": 16,
             "CX": 64, "CZ": 65, "SWAP": 66, "RZZ": 67, "MAT2": 68}


class Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint16), ("reserved", ctypes.c_uint16), ("q", ctypes.c_int32 * 2),
                ("theta", ctypes.c_double * 3), ("param_idx", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("mat", ctypes.POINTER(ctypes.c_double))]


class PauliTerm(ctypes.Structure):
    _fields_ = [("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64), ("coeff", ctypes.c_double)]


class NoiseModel(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("flags", ctypes.c_uint32), ("T1_us", ctypes.POINTER(ctypes.c_double)),
                ("T2_us", ctypes.POINTER(ctypes.c_double)), ("t1q_ns", ctypes.c_double),
                ("t2q_ns", ctypes.c_double), ("p1", ctypes.c_double), ("p2", ctypes.c_double),
                ("readout_e", ctypes.c_double)]


class PlanTuning(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int32), ("fusion_bits", ctypes.c_int32), ("register_bits", ctypes.c_int32)]

    def as_dict(self):
        return dict(tile_bits=self.tile_bits, fusion_bits=self.fusion_bits, register_bits=self.register_bits)


class BatchTemplate(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("gates", ctypes.POINTER(Gate)), ("ngates", ctypes.c_size_t),
                ("terms", ctypes.POINTER(PauliTerm)), ("nterms", ctypes.c_size_t),
                ("coeffs", ctypes.POINTER(ctypes.c_double)), ("ne", ctypes.c_int32)]


class NwqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nwq error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libnwqgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2401_06861_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, i32, u32, dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
    P = ctypes.POINTER
    pp = P(ctypes.c_void_p)
    sig = {
        "nwq_state_bytes": (sz, [i32, i32, i32]),
        "nwq_sv_create": (i32, [i32, i32, vp, sz, vp, pp]),
        "nwq_dm_create": (i32, [i32, i32, vp, sz, vp, pp]),
        "nwq_state_reset": (i32, [vp]),
        "nwq_state_load": (i32, [vp, vp, sz, i32]),
        "nwq_state_copy": (i32, [vp, vp, sz, i32]),
        "nwq_dm_copy_pauli": (i32, [vp, vp, sz, i32]),
        "nwq_dm_load_pauli": (i32, [vp, vp, sz, i32]),
        "nwq_destroy": (i32, [vp]),
        "nwq_sv_apply_circuit": (i32, [vp, P(Gate), sz, u32]),
        "nwq_dm_apply_circuit_noisy": (i32, [vp, P(Gate), sz, P(NoiseModel), u32]),
        "nwq_plan_create": (i32, [i32, i32, i32, P(Gate), sz, P(NoiseModel), u32, vp, pp]),
        "nwq_plan_run": (i32, [vp, vp]),
        "nwq_plan_info": (i32, [vp, P(i32), P(i32), P(dbl), P(dbl), P(sz)]),
        "nwq_plan_layout": (i32, [vp, P(i32), P(i32), P(i32)]),
        "nwq_plan_destroy": (i32, [vp]),
        "nwq_plan_create_tuned": (i32, [i32, i32, i32, P(Gate), sz, P(NoiseModel), u32, P(PlanTuning), vp, pp]),
        "nwq_plan_autotune": (i32, [vp, P(Gate), sz, P(NoiseModel), u32, i32, P(PlanTuning), P(dbl),
                                    P(PlanTuning), P(dbl), i32, P(i32)]),
        "nwq_plan_jit_check": (i32, [vp, P(i32), P(i32)]),
        "nwq_plan_verify": (i32, [vp]),
        "nwq_plan_tc_blocks": (i32, [vp, P(i32), P(dbl)]),
        "nwq_plan_ops": (i32, [vp, P(i32), P(i32), P(dbl)]),
        "nwq_expect_plan": (i32, [i32, P(PauliTerm), sz, i32, P(i32), P(ctypes.c_uint64), P(i32),
                                  P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint64), P(i32), P(i32),
                                  P(i32), P(i32)]),
        "nwq_tc_timeouts": (i32, [P(i32)]),
        "nwq_tc_wait_test": (i32, [vp, vp, P(i32)]),
        "nwq_plan_jit_prefetch": (i32, [vp, P(i32)]),
        "nwq_plan_kernel_arith": (i32, [vp, i32, P(dbl), P(dbl), P(dbl), P(i32)]),
        "nwq_plan_last_run_dw": (i32, [vp, P(i32)]),
        "nwq_jit_shutdown": (i32, []),
        "nwq_expect_pauli_sum": (i32, [vp, P(PauliTerm), sz, P(dbl), u32]),
        "nwq_expect_pauli_sum_noalloc": (i32, [vp, P(PauliTerm), sz, P(dbl), u32]),
        "nwq_expect_launch_shape": (i32, [vp, sz, i32, P(i32), P(i32)]),
        "nwq_probs": (i32, [vp, dbl, P(dbl)]),
        "nwq_batch_energy": (i32, [i32, i32, P(Gate), sz, vp, i32, i32, P(PauliTerm), sz, P(dbl), i32, vp, vp]),
        "nwq_batch_create": (i32, [i32, P(BatchTemplate), i32, i32, vp, pp]),
        "nwq_batch_run": (i32, [vp, vp, vp, i32, vp, i32, vp, vp, u32]),
        "nwq_batch_destroy": (i32, [vp]),
        "nwq_batch_set_shape": (i32, [vp, i32, i32]),
        "nwq_traj_draws": (i32, [P(Gate), sz, i32, P(NoiseModel), P(sz)]),
        "nwq_traj_run": (i32, [i32, i32, P(Gate), sz, P(NoiseModel), P(PauliTerm), sz, P(dbl), i32, vp, i32, vp, vp]),
        "nwq_batch_autotune": (i32, [vp, vp, vp, i32, vp, i32, i32, vp, P(i32), P(i32), P(dbl)]),
        "nwq_last_error": (ctypes.c_char_p, []),
        "nwq_device_sync": (i32, [vp]),
        "nwq_launch_count": (ctypes.c_uint64, []),
        "nwq_peak_probe": (i32, [i32, P(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    # stop the library's background kernel compiler while the interpreter is
    # still alive, before any C-level exit handler tears its dependencies down
    atexit.register(L.nwq_jit_shutdown)
    return L


def check(rc):
    if rc != OK:
        raise NwqError(rc, lib().nwq_last_error().decode())
    return rc


# ------------------------------------------------------------------ marshalling
# numpy mirror of nwq_gate (56 bytes) for vectorised marshalling
GATE_DTYPE = np.dtype({"names": ["kind", "reserved", "q", "theta", "param_idx", "reserved2", "mat"],
                       "formats": [np.uint16, np.uint16, (np.int32, 2), (np.float64, 3), np.int32, np.int32,
                                   np.uint64],
                       "offsets": [0, 2, 4, 16, 40, 44, 48], "itemsize": 56})


def encode_gates_np(gates, param_index=None):
    """Gate tuples -> numpy array laid out as nwq_gate[] (plus keep-alive list).
    Column-wise; MAT1/MAT2 matrices are pointed to by address."""
    ng = len(gates)
    a = np.zeros(max(ng, 1), GATE_DTYPE)
    if ng == 0:
        return a, []
    a["kind"][:ng] = np.fromiter((GATE_KIND[g[0]] for g in gates), np.uint16, ng)
    a["q"][:ng, 0] = np.fromiter((g[1][0] for g in gates), np.int32, ng)
    a["q"][:ng, 1] = np.fromiter((g[1][1] if len(g[1]) > 1 else 0 for g in gates), np.int32, ng)
    keep = []
    mats = [i for i, g in enumerate(gates) if g[0].startswith("MAT")]
    if len(mats) < ng:
        a["theta"][:ng] = np.array([(tuple(g[2]) + (0.0, 0.0, 0.0))[:3] if not g[0].startswith("MAT") else (0.0, 0.0, 0.0)
                                    for g in gates], np.float64)
    for i in mats:
        m = np.ascontiguousarray(np.asarray(gates[i][2], np.complex128)).view(np.float64).copy()
        keep.append(m)
        a["mat"][i] = m.ctypes.data
    a["param_idx"][:ng] = -1 if param_index is None else np.asarray(param_index, np.int32)
    return a, keep


def encode_gates(gates, param_index=None):
    """Gate tuples (name, qubits, params) -> (ctypes array, keep-alive list)."""
    arr = (Gate * max(len(gates), 1))()
    keep = []
    for i, (name, qs, prm) in enumerate(gates):
        g = arr[i]
        g.kind = GATE_KIND[name]
        for j, q in enumerate(qs):
            g.q[j] = q
        g.param_idx = -1 if param_index is None else int(param_index[i])
        if name.startswith("MAT"):
            m = np.ascontiguousarray(np.asarray(prm, np.complex128)).view(np.float64).copy()
            keep.append(m)
            g.mat = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            for j, p in enumerate(prm):
                g.theta[j] = p
    return arr, keep


def encode_terms(terms):
    arr = (PauliTerm * max(len(terms), 1))()
    for i, (x, z, c) in enumerate(terms):
        arr[i].x_mask, arr[i].z_mask, arr[i].coeff = int(x), int(z), float(c)
    return arr


def encode_noise(noise, n):
    if noise is None:
        return None, []
    T1 = np.ascontiguousarray(noise["T1_us"], np.float64)
    T2 = np.ascontiguousarray(noise["T2_us"], np.float64)
    nm = NoiseModel()
    nm.n = min(len(T1), len(T2))
    nm.flags = (NOISE_RZ_VIRTUAL if noise.get("rz_virtual") else 0) | \
               (NOISE_DEPOL_PAULI_FORM if noise.get("depol_pauli_form") else 0)
    nm.T1_us = T1.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nm.T2_us = T2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nm.t1q_ns, nm.t2q_ns = noise["t1q_ns"], noise["t2q_ns"]
    nm.p1, nm.p2, nm.readout_e = noise["p1"], noise["p2"], noise["readout_e"]
    return nm, [T1, T2]
