"""Thin Python layer over the C ABI (same names, numpy in and out).

    st = State(SV, n, F64)            # nwq_sv_create
    st.apply(gates)                   # nwq_sv_apply_circuit
    st.expect(terms)                  # nwq_expect_pauli_sum
    st.probs(readout_e)               # nwq_probs
    st.copy()                         # nwq_state_copy

Device memory may be library-owned (default) or a caller buffer such as a
torch tensor (``buf=tensor.data_ptr(), buf_bytes=...``).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np

from . import _lib as L
from ._lib import DM, F32, F64, SV, check, encode_gates, encode_noise, encode_terms  # noqa: F401


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def state_bytes(kind, n, dtype):
    return L.lib().nwq_state_bytes(kind, n, dtype)


def launch_count():
    """Kernels launched so far by the CUDA library in this process."""
    return int(L.lib().nwq_launch_count())


class State:
    def __init__(self, kind, n, dtype=F64, buf=None, buf_bytes=0, stream=None):
        self.kind, self.n, self.dtype = kind, n, dtype
        self.h = ctypes.c_void_p()
        create = L.lib().nwq_sv_create if kind == SV else L.lib().nwq_dm_create
        check(create(n, dtype, ctypes.c_void_p(buf) if buf else None, buf_bytes,
                     ctypes.c_void_p(stream) if stream else None, ctypes.byref(self.h)))

    # -- lifetime
    def close(self):
        if self.h:
            L.lib().nwq_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- circuits
    def apply(self, gates, noise=None, flags=0):
        arr, keep = encode_gates(gates)
        if self.kind == SV:
            check(L.lib().nwq_sv_apply_circuit(self.h, arr, len(gates), flags))
        else:
            nm, keep2 = encode_noise(noise, self.n)
            check(L.lib().nwq_dm_apply_circuit_noisy(self.h, arr, len(gates),
                                                      ctypes.byref(nm) if nm is not None else None, flags))
        return self

    def apply_encoded(self, arr, ng, noise=None, flags=0):
        """apply() from an ``_lib.encode_gates_np`` array (one-shot lowering)."""
        g = ctypes.cast(ctypes.c_void_p(arr.ctypes.data), ctypes.POINTER(L.Gate))
        if self.kind == SV:
            check(L.lib().nwq_sv_apply_circuit(self.h, g, ng, flags))
        else:
            nm, keep2 = encode_noise(noise, self.n)
            check(L.lib().nwq_dm_apply_circuit_noisy(self.h, g, ng, ctypes.byref(nm) if nm is not None else None,
                                                      flags))
        return self

    def run(self, plan):
        check(L.lib().nwq_plan_run(self.h, plan.h))
        return self

    def reset(self):
        check(L.lib().nwq_state_reset(self.h))

    def sync(self):
        check(L.lib().nwq_device_sync(self.h))

    # -- measurement
    def expect(self, terms, sum=False, normalize=False):
        """Per-term <P> (or sum_t coeff_t <P_t> with sum=True); normalize=True
        divides by the FP64 norm (SV) / trace (DM) of the state."""
        arr = encode_terms(terms)
        out = np.zeros(1 if sum else max(len(terms), 1))
        flags = (L.EXPECT_SUM if sum else L.EXPECT_TERMS) | (L.EXPECT_NORMALIZE if normalize else 0)
        check(L.lib().nwq_expect_pauli_sum(self.h, arr, len(terms), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           flags))
        return float(out[0]) if sum else out[:len(terms)]

    def norm(self):
        """<psi|psi> (SV) or Tr(rho) (DM), accumulated in FP64."""
        return float(self.expect([(0, 0, 1.0)])[0])

    def probs(self, readout_e=0.0):
        out = np.zeros(1 << self.n)
        check(L.lib().nwq_probs(self.h, float(readout_e), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    # -- state transfer
    def _cdtype(self):
        return np.complex128 if self.dtype == F64 else np.complex64

    def copy(self):
        """SV: amplitudes.  DM: rho as a row-major (2^n, 2^n) matrix."""
        N = 1 << self.n
        if self.kind == SV:
            out = np.zeros(N, self._cdtype())
        else:
            out = np.zeros(N * N, self._cdtype())
        check(L.lib().nwq_state_copy(self.h, _ptr(out), out.nbytes, 0))
        if self.kind == DM:
            return out.reshape(N, N).T.copy()
        return out

    def pauli(self):
        out = np.zeros(1 << (2 * self.n), np.float64 if self.dtype == F64 else np.float32)
        check(L.lib().nwq_dm_copy_pauli(self.h, _ptr(out), out.nbytes, 0))
        return out

    def load_pauli(self, coeffs):
        """DM: load raw Pauli-basis coefficients (as ``pauli()`` returns them)."""
        a = np.ascontiguousarray(coeffs, np.float64 if self.dtype == F64 else np.float32)
        check(L.lib().nwq_dm_load_pauli(self.h, _ptr(a), a.nbytes, 0))

    def load(self, data):
        """SV: amplitude vector.  DM: row-major rho matrix."""
        if self.kind == SV:
            a = np.ascontiguousarray(data, self._cdtype())
        else:
            a = np.ascontiguousarray(np.asarray(data).T, self._cdtype()).reshape(-1)
        check(L.lib().nwq_state_load(self.h, _ptr(a), a.nbytes, 0))


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, L.PlanTuning):
        return t
    return L.PlanTuning(int(t.get("tile_bits", 0)), int(t.get("fusion_bits", 0)), int(t.get("register_bits", 0)))


def expect_plan(n, terms, normalize=False):
    """The pass plan of nwq_expect_pauli_sum (host only): dict(passes=[(tile mask,
    [(out, xl, zl, zh, y), ...]), ...], general=[term index, ...])."""
    nt = len(terms)
    arr = encode_terms(terms)
    m = nt + 1
    P32, P64 = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64)
    npass, nfb = ctypes.c_int(), ctypes.c_int()
    tiles = np.zeros(m, np.uint64)
    rng = np.zeros(2 * m, np.int32)
    xl, zl = np.zeros(m, np.uint32), np.zeros(m, np.uint32)
    zh = np.zeros(m, np.uint64)
    y, out, fb = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m, np.int32)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    check(L.lib().nwq_expect_plan(n, arr, nt, int(normalize), ctypes.byref(npass), tiles.ctypes.data_as(P64),
                                  rng.ctypes.data_as(P32), xl.ctypes.data_as(u32), zl.ctypes.data_as(u32),
                                  zh.ctypes.data_as(P64), y.ctypes.data_as(P32), out.ctypes.data_as(P32),
                                  ctypes.byref(nfb), fb.ctypes.data_as(P32)))
    passes = []
    for p in range(npass.value):
        k0, nk = int(rng[2 * p]), int(rng[2 * p + 1])
        passes.append((int(tiles[p]), [(int(out[r]), int(xl[r]), int(zl[r]), int(zh[r]), int(y[r]))
                                       for r in range(k0, k0 + nk)]))
    return dict(passes=passes, general=[int(v) for v in fb[:nfb.value]])


def tc_timeouts():
    """Bounded waits of the tensor-core kernel that ran out on the current device (0 when healthy)."""
    c = ctypes.c_int()
    check(L.lib().nwq_tc_timeouts(ctypes.byref(c)))
    return c.value


def _device_name():
    try:
        import torch
        return torch.cuda.get_device_name() if torch.cuda.is_available() else "no-device"
    except Exception:  # torch is optional plumbing
        return "unknown-device"


def autotune_key(kind, n, dtype, gates, noise=None, flags=0, device=None):
    """Cache key of an autotuning result: the device name and the circuit's
    structure (kind, qubits, precision, flags, noise or not, each gate's kind
    and qubits); angles and matrices are left out, as they do not change
    which plan shape runs fastest."""
    desc = [device if device is not None else _device_name(), int(kind), int(n), int(dtype), int(flags),
            noise is not None, [(g[0], [int(q) for q in g[1]]) for g in gates]]
    return hashlib.sha256(json.dumps(desc, separators=(",", ":")).encode()).hexdigest()


def autotune(state, gates, noise=None, flags=0, reps=3, cache=None):
    """Time the circuit's plan for each candidate shape on ``state`` (a State
    of the circuit's kind, size and dtype; overwritten) and return
    dict(best=tuning dict, best_ms, tried=[(tuning dict, ms)]).

    ``cache``: a JSON file of earlier results (default: the file named by the
    environment variable NWQ_AUTOTUNE_CACHE, none if unset), keyed by
    ``autotune_key``.  A hit returns the stored result (with cached=True)
    without running anything; a miss runs the tuner and adds its result."""
    path = cache if cache is not None else os.environ.get("NWQ_AUTOTUNE_CACHE")
    key = data = None
    if path:
        key = autotune_key(state.kind, state.n, state.dtype, gates, noise, flags)
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
        if key in data:
            return dict(data[key], cached=True)
    arr, keep = encode_gates(gates)
    nm, keep2 = encode_noise(noise, state.n)
    best, bms = L.PlanTuning(), ctypes.c_double()
    tried, tms, nt = (L.PlanTuning * 32)(), (ctypes.c_double * 32)(), ctypes.c_int()
    check(L.lib().nwq_plan_autotune(state.h, arr, len(gates), ctypes.byref(nm) if nm is not None else None, flags,
                                    reps, ctypes.byref(best), ctypes.byref(bms), tried, tms, 32, ctypes.byref(nt)))
    res = dict(best=best.as_dict(), best_ms=bms.value,
               tried=[(tried[i].as_dict(), tms[i]) for i in range(nt.value)])
    if path:
        data[key] = res
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f)
        os.replace(tmp, path)
    return dict(res, cached=False)


class Plan:
    def __init__(self, kind, n, gates, dtype=F64, noise=None, flags=0, encoded=None, tuning=None):
        """Lower ``gates`` (tuples), or an ``encoded`` nwq_gate array from
        ``_lib.encode_gates_np``, once for repeated runs; ``tuning`` (a dict
        of tile_bits / fusion_bits / register_bits, e.g. ``autotune(...)["best"]``)
        fixes the plan shape."""
        if encoded is None:
            arr, keep = encode_gates(gates)
            ng = len(gates)
        else:
            arr = ctypes.cast(ctypes.c_void_p(encoded.ctypes.data), ctypes.POINTER(L.Gate))
            ng = len(encoded) if gates is None else len(gates)
        nm, keep2 = encode_noise(noise, n)
        self.h = ctypes.c_void_p()
        tu = _tuning(tuning)
        check(L.lib().nwq_plan_create_tuned(kind, n, dtype, arr, ng, ctypes.byref(nm) if nm is not None else None,
                                            flags, ctypes.byref(tu) if tu is not None else None, None,
                                            ctypes.byref(self.h)))
        self.ngates = ng

    def info(self):
        s, o = ctypes.c_int(), ctypes.c_int()
        b, f = ctypes.c_double(), ctypes.c_double()
        tb = ctypes.c_size_t()
        check(L.lib().nwq_plan_info(self.h, ctypes.byref(s), ctypes.byref(o), ctypes.byref(b), ctypes.byref(f),
                                    ctypes.byref(tb)))
        return dict(sweeps=s.value, ops=o.value, bytes=b.value, fma_per_elem=f.value, table_bytes=tb.value)

    def layout(self):
        info = self.info()
        sw = (ctypes.c_int * max(info["sweeps"], 1))()
        og = (ctypes.c_int * max(info["ops"], 1))()
        on = (ctypes.c_int * max(info["ops"], 1))()
        check(L.lib().nwq_plan_layout(self.h, sw, og, on))
        return list(sw)[:info["sweeps"]], list(og)[:info["ops"]], list(on)[:info["ops"]]

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def verify(self):
        """Check the plan's device tables against the kernels' bounds (raises NwqError)."""
        check(L.lib().nwq_plan_verify(self.h))

    def ops(self):
        """Merged operators of a sweep plan in execution order: list of
        (index bits, 2^k x 2^k complex matrix), local index bit t <-> bits[t]
        (qubits for state vectors; Pauli-coefficient index bits, real
        matrices, for density matrices)."""
        no = self.info()["ops"]
        k = np.zeros(max(no, 1), np.int32)
        bits = np.zeros(max(no, 1) * 4, np.int32)
        ms = np.zeros(max(no, 1) * 512, np.float64)
        check(L.lib().nwq_plan_ops(self.h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   bits.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        mats = ms.view(np.complex128).reshape(-1, 16, 16)
        out = []
        for o in range(no):
            d = 1 << int(k[o])
            out.append((tuple(int(b) for b in bits[4 * o:4 * o + int(k[o])]), mats[o, :d, :d].copy()))
        return out

    def tc_blocks(self):
        """Blocks of a tensor-core plan (flags=PLAN_TC): list of (qubits, 32x32 complex matrix)."""
        nb = self.info()["sweeps"]
        qs = np.zeros(max(nb, 1) * 5, np.int32)
        ms = np.zeros(max(nb, 1) * 2048, np.float64)
        check(L.lib().nwq_plan_tc_blocks(self.h, qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        mats = ms.view(np.complex128).reshape(-1, 32, 32)
        return [(tuple(int(q) for q in qs[5 * b:5 * b + 5]), mats[b].copy()) for b in range(nb)]

    def kernel_arith(self, dw=False):
        """Per state element, summed over the sweeps with specialised kernels:
        (multiply-adds, multiplies, arithmetic-pipe instructions, sweeps) as
        generated (dw: the double-word kernels of an FP64 plan, whose
        instructions are FP32 ones)."""
        f, m, i, sw = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        check(L.lib().nwq_plan_kernel_arith(self.h, 1 if dw else 0, ctypes.byref(f), ctypes.byref(m),
                                            ctypes.byref(i), ctypes.byref(sw)))
        return f.value, m.value, i.value, sw.value

    def last_run_dw(self):
        """True when the latest run took the double-word path."""
        d = ctypes.c_int()
        check(L.lib().nwq_plan_last_run_dw(self.h, ctypes.byref(d)))
        return bool(d.value)

    def jit_check(self):
        """Compile (host only) the specialised kernels of this plan's sweeps:
        returns (eligible sweeps, compiled sweeps)."""
        e, b = ctypes.c_int(), ctypes.c_int()
        check(L.lib().nwq_plan_jit_check(self.h, ctypes.byref(e), ctypes.byref(b)))
        return e.value, b.value

    def jit_prefetch(self):
        """Queue background compilation of this plan's specialised kernels;
        returns the number pending (does not wait)."""
        q = ctypes.c_int()
        check(L.lib().nwq_plan_jit_prefetch(self.h, ctypes.byref(q)))
        return q.value

    def close(self):
        if self.h:
            L.lib().nwq_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched parametrised circuits (nwq_batch_create / nwq_batch_run).

    templates: list of dicts {n, gates, param_index, terms, coeffs (ne x nt)}.
    run(params, out, job_template=None, norms=None): device tensors (torch or
    raw pointers); asynchronous on ``stream``.
    """

    def __init__(self, templates, nparams, dtype=F64, stream=None):
        self.keep = []
        arr = (L.BatchTemplate * len(templates))()
        self.max_ne = 0
        for i, t in enumerate(templates):
            ga, k1 = L.encode_gates_np(t["gates"], t.get("param_index"))
            g = ctypes.cast(ctypes.c_void_p(ga.ctypes.data), ctypes.POINTER(L.Gate))
            k1 = (ga, k1)
            tr = encode_terms(t["terms"])
            c = np.ascontiguousarray(t["coeffs"], np.float64).reshape(-1)
            ne = int(np.asarray(t["coeffs"]).reshape(-1, max(len(t["terms"]), 1)).shape[0]) if len(t["terms"]) else 1
            self.keep += [g, k1, tr, c]
            arr[i].n = t["n"]
            arr[i].gates = g
            arr[i].ngates = len(t["gates"])
            arr[i].terms = ctypes.cast(tr, ctypes.POINTER(L.PauliTerm))
            arr[i].nterms = len(t["terms"])
            arr[i].coeffs = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[i].ne = ne
            self.max_ne = max(self.max_ne, ne)
        self.h = ctypes.c_void_p()
        check(L.lib().nwq_batch_create(dtype, arr, len(templates), nparams,
                                       ctypes.c_void_p(stream) if stream else None, ctypes.byref(self.h)))
        self.keep = None

    def run(self, params_ptr, njobs, out_ptr, out_stride=None, job_template_ptr=None, norms_ptr=None,
            stream=None, graph=False, fp64_pipe=False):
        """fp64_pipe: FP64 batches on the FP64 pipe instead of double words."""
        flags = (L.BATCH_GRAPH if graph else 0) | (L.BATCH_FP64_PIPE if fp64_pipe else 0)
        check(L.lib().nwq_batch_run(self.h, ctypes.c_void_p(params_ptr), ctypes.c_void_p(job_template_ptr)
                                    if job_template_ptr else None, njobs, ctypes.c_void_p(out_ptr),
                                    out_stride or self.max_ne, ctypes.c_void_p(norms_ptr) if norms_ptr else None,
                                    ctypes.c_void_p(stream) if stream else None, flags))

    def set_shape(self, threads=256, fusion=0):
        """Threads per CTA (128 / 256 / 512) and gate-fusion width (0 / 1)."""
        check(L.lib().nwq_batch_set_shape(self.h, threads, fusion))

    def autotune(self, params_ptr, njobs, out_ptr, out_stride=None, job_template_ptr=None, reps=3, stream=None):
        """Time every kernel shape on these jobs, keep the fastest; returns
        dict(threads, fusion, ms)."""
        th, fu, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(L.lib().nwq_batch_autotune(self.h, ctypes.c_void_p(params_ptr),
                                         ctypes.c_void_p(job_template_ptr) if job_template_ptr else None, njobs,
                                         ctypes.c_void_p(out_ptr), out_stride or self.max_ne, reps,
                                         ctypes.c_void_p(stream) if stream else None, ctypes.byref(th),
                                         ctypes.byref(fu), ctypes.byref(ms)))
        return dict(threads=th.value, fusion=fu.value, ms=ms.value)

    def close(self):
        if self.h:
            L.lib().nwq_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trajectory_draws(n, gates, noise):
    """Uniform draws one quantum trajectory of ``gates`` under ``noise`` consumes."""
    arr, keep = encode_gates(gates)
    nm, keep2 = encode_noise(noise, n)
    d = ctypes.c_size_t()
    check(L.lib().nwq_traj_draws(arr, len(gates), n, ctypes.byref(nm) if nm is not None else None, ctypes.byref(d)))
    return d.value


def trajectories(n, gates, noise, terms, coeffs, ntraj, dtype=F64, seed=0, uniforms=None, stream=None):
    """Noisy energies by quantum trajectories (nwq_traj_run): returns an
    (ntraj, ne) array, row t = sum_k coeffs[e, k] <P_k> of trajectory t.  The
    draws are ``uniforms`` (ntraj x draws, in [0, 1)) or, by default, numpy's
    default_rng(seed)."""
    import torch
    arr, keep = encode_gates(gates)
    nm, keep2 = encode_noise(noise, n)
    d = trajectory_draws(n, gates, noise)
    if uniforms is None:
        uniforms = np.random.default_rng(seed).random((ntraj, d))
    u = torch.from_numpy(np.ascontiguousarray(uniforms, np.float64).reshape(ntraj, d)).cuda()
    c = np.ascontiguousarray(np.asarray(coeffs, np.float64).reshape(-1, len(terms)))
    ne = c.shape[0]
    out = torch.empty(ntraj, ne, dtype=torch.float64, device="cuda")
    tr = encode_terms(terms)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    check(L.lib().nwq_traj_run(n, dtype, arr, len(gates), ctypes.byref(nm) if nm is not None else None, tr, len(terms),
                               c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ne,
                               ctypes.c_void_p(u.data_ptr() if d else 0), ntraj, ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(s)))
    return out.cpu().numpy()
