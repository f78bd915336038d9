"""Benchmark of the hot path of NWQ-Sim's simulators (paper Sec. II-III) on one GB300.

Default line: the largest single-GPU state-vector workload.  Transverse-field
Ising chain, n = 33 qubits in complex128 (a 128 GiB state), 10 first-order
Trotter steps (J = 1, dt = 0.05, per-qubit fields h_i ~ U(0.5, 2) from seed
3334; per step CX RZ(2 J dt) CX on the 32 bonds, then RX(2 h_i dt) on every
qubit: 1290 gates), run as one reusable fused plan.  One step = reset to
|0..0>  ->  the whole circuit  ->  <Z_i> for every qubit and <H> (FP64 sums).
Metric: gate-updates/s = sum over the original (unfused) gates of the
amplitudes each logically updates (2^n per one-qubit or diagonal gate,
2^(n-1) per CX), per second.

--workload dm: the noisy density-matrix TFIM (n = 13, 20 Trotter steps,
FP64): reset rho -> 980 gates, each followed by depolarising and thermal
relaxation -> <Z_i>, <H> -> the outcome distribution with 2% readout error;
gate-updates = gates x 4^n.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload sv|dm|...]
Under torchrun each rank runs its own replica (independent problems, weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate-updates/s"
UNIT = "gate-updates/s"
_CSRC = os.path.join(ROOT, "paper_2401_06861_gb300", "csrc")

# ---- the large state-vector workload (default)
SV_N, SV_DEPTH = 33, 10
SV_WORKLOAD = f"sv_tfim_n{SV_N}_c128_depth{SV_DEPTH}"
SV_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sv_jit_sweep_c128_n33_traffic.json")
SV_KERNEL = "nwq_jit_sweep (run-time specialised complex128 sweep)"
SV_KERNEL_DW = "nwq_jit_sweep (run-time specialised complex128 sweep, double-word arithmetic)"
SV_TRAFFIC_FILE_DW = os.path.join(ROOT, "profiles", "sv_jit_sweep_dw_n33_traffic.json")

# ---- the noisy density-matrix workload (--workload dm)
N = 13
TROTTER_STEPS = 20
WORKLOAD = f"dm_noisy_tfim_n{N}_{TROTTER_STEPS}steps"
# The DM sweeps run the run-time specialised kernel (generated by jit.cpp from
# the plan of planner.cpp) unless NWQ_JIT=0 selects the interpreted one.
JIT = os.environ.get("NWQ_JIT", "1") != "0"
JIT_SRCS = [os.path.join(_CSRC, f) for f in ("jit.cpp", "planner.cpp")]
if JIT:
    KERNEL_SRCS = JIT_SRCS
    TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dm_jit_sweep_f64_n13_traffic.json")
    KERNEL_NAME = "nwq_jit_sweep (run-time specialised FP64 Pauli-basis DM sweep)"
    KERNEL_NAME_DW = "nwq_jit_sweep (run-time specialised Pauli-basis DM sweep, double-word arithmetic)"
    TRAFFIC_FILE_DW = os.path.join(ROOT, "profiles", "dm_jit_sweep_dw_n13_traffic.json")
else:
    KERNEL_SRCS = [os.path.join(_CSRC, f) for f in ("sweep_kernels.cu", "device_util.cuh")]
    TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dm_sweep_f64_n13_traffic.json")
    KERNEL_NAME = "sweep_kernel<double,real> (FP64 Pauli-basis DM sweep, interpreted)"
    KERNEL_NAME_DW, TRAFFIC_FILE_DW = KERNEL_NAME, TRAFFIC_FILE


def workload():
    from paper_2401_06861_gb300 import inputs
    gates, noise = inputs.dm_noisy_tfim(N, TROTTER_STEPS)
    return gates, noise, inputs.z_terms(N), inputs.tfim_terms(N)


def sv_workload(n=SV_N, depth=SV_DEPTH):
    from paper_2401_06861_gb300 import inputs
    gates, h = inputs.large_sv_tfim(n, depth)
    return gates, h, inputs.z_terms(n), inputs.tfim_terms(n, 1.0, h)


def sv_gate_updates(gates, n):
    """Amplitudes the original gates logically update: 2^(n-1) per CX (the
    control = 1 half moves), 2^n per other gate."""
    return sum(2.0 ** (n - 1) if g[0] == "CX" else 2.0 ** n for g in gates)


def config_of(workload_name, ws):
    """The workload description printed by both arms."""
    if workload_name == "sv":
        return {"workload": SV_WORKLOAD, "n": SV_N, "state": "complex128 (16 B/amplitude, 128 GiB)",
                "gates": SV_DEPTH * (3 * (SV_N - 1) + SV_N), "trotter_steps": SV_DEPTH, "J": 1.0, "dt": 0.05,
                "h": "U(0.5, 2), seed 3334", "l2": "inputs larger than L2 (128 GiB state)",
                "parallelism": f"replicas x{ws}"}
    return {"workload": WORKLOAD, "n": N, "gates": TROTTER_STEPS * (3 * (N - 1) + N), "trotter_steps": TROTTER_STEPS,
            "state_bytes": 8 << (2 * N), "l2": "inputs larger than L2 (512 MiB state)",
            "noise": "depolarising p1=1e-3 / p2=1e-2, relaxation 35 / 300 ns, T1/T2 seed 2401, readout 2%",
            "parallelism": f"replicas x{ws}"}


def reduce_max(x, ws):
    """Max over ranks of a host float (the slowest rank sets the job's time)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, seconds):
    """Whole-job throughput: every rank processed units_per_rank in `seconds`
    (the max over ranks)."""
    return units_per_rank * ws / seconds


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("NWQ_BENCH_BACKEND") != "gloo" else "gloo")
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region (200 ms period)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.p = None
        self.device = device
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def traffic_per_launch(path, srcs):
    """DRAM bytes per sweep launch from a committed ncu summary, or None if the
    kernel sources changed since the counters were taken."""
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(b"".join(open(f, "rb").read() for f in srcs)).hexdigest()[:16]
        return rec["traffic_bytes_per_launch"] if rec.get("kernel_sha") == h else None
    except (OSError, ValueError, KeyError):
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "fallback": True}


def probe_rate(what):
    """FMA instructions per second of one pipe, measured now (nwq_peak_probe)."""
    import ctypes

    from paper_2401_06861_gb300 import _lib as L
    v = ctypes.c_double(0.0)
    L.check(L.lib().nwq_peak_probe(what, ctypes.byref(v)))
    return v.value


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(gates, noise, ngates):
    """Time the CPU oracle on the first ``ngates`` noisy gates of the DM workload."""
    import oracle
    oracle.lib()
    t0 = time.perf_counter()
    oracle.dm_run(N, gates[:ngates], noise)
    dt = time.perf_counter() - t0
    return ngates * 4.0 ** N / dt, dt


def cpu_cores():
    try:
        aff = len(os.sched_getaffinity(0))
    except AttributeError:
        aff = os.cpu_count()
    return int(os.environ.get("OMP_NUM_THREADS", aff))


def oracle_sv_rate(n, gates, threads):
    """Gate-updates/s of the oracle on ``gates`` from |0..0> at n qubits with
    ``threads`` OpenMP threads, and the seconds it took."""
    import oracle
    oracle.set_threads(threads)
    psi = oracle.zero_state(n)
    t0 = time.perf_counter()
    oracle.sv_run_inplace(psi, n, gates)
    dt = time.perf_counter() - t0
    del psi
    return sv_gate_updates(gates, n) / dt, dt


def sv_cpu_baseline():
    """The oracle (plain FP64 C, OpenMP over amplitude groups) on the same
    circuit family: one Trotter step at n = 26 on all host cores and at n = 22
    on one core.  The per-amplitude work of a gate does not depend on n once
    the state is far larger than the CPU caches, so the rate stands for the
    n = 33 workload (whose 10 steps would take that time x 2^(33-26) x 10)."""
    cores = cpu_cores()
    g26 = sv_workload(26, 1)[0]
    g22 = sv_workload(22, 1)[0]
    v_all, t_all = oracle_sv_rate(26, g26, cores)
    v_one, t_one = oracle_sv_rate(22, g22, 1)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one Trotter step of the same chain ({len(g26)} gates) at n=26 (1 GiB complex128) on "
                      f"{cores} threads, {t_all:.1f} s; same at n=22 on 1 thread: {v_one:.3e} {UNIT} "
                      f"({t_one:.1f} s); n=33 x 10 steps would take {t_all * 2 ** 7 * 10:.0f} s at this rate",
            "single_thread_value": v_one}


def sv_oracle_check(gates, h, z, zz, x, e):
    """The GPU results against the exact free-fermion values of the same
    circuit (oracle/tfim_fermion.py): max term error and relative energy error."""
    import numpy as np

    from oracle import tfim_fermion
    ref = tfim_fermion.tfim_observables(SV_N, gates)
    eref = -float(np.sum(ref["zz"])) - float(np.dot(h, ref["x"]))
    norm1 = (SV_N - 1) + float(np.sum(np.abs(h)))
    return {"max_term_err": float(max(np.max(np.abs(zz - ref["zz"])), np.max(np.abs(x - ref["x"])),
                                      abs(z[0] - ref["z0"]))),
            "rel_energy_err": abs(e - eref) / max(abs(eref), norm1), "energy_exact": eref,
            "reference": "free-fermion values of <Z_i Z_i+1>, <X_i>, <Z_0> (oracle/tfim_fermion.py)"}


def run_reference(args, ws, rank):
    """The oracle as the reference arm, on host cores, bounded samples per step."""
    if rank != 0:
        return 0
    cores = cpu_cores()
    if args.workload == "dm":
        gates, noise, _, _ = workload()
        vals = []
        for i in range(args.warmup + args.steps):
            v, _ = oracle_sample(gates, noise, 1)
            if i >= args.warmup:
                vals.append(v)
        value = statistics.mean(vals)
        sample = f"first noisy gate (CX(0,1) + 2q depolarising + relaxation) of the n={N} circuit, per step"
        ms = 4.0 ** N / value * 1e3
    else:
        import oracle
        oracle.set_threads(cores)
        n, per = 26, 12
        g = sv_workload(n, 1)[0]
        psi = oracle.zero_state(n)
        upd = tm = 0.0
        for i in range(args.warmup + args.steps):
            sl = [g[(i * per + j) % len(g)] for j in range(per)]
            t0 = time.perf_counter()
            oracle.sv_run_inplace(psi, n, sl)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                upd += sv_gate_updates(sl, n)
                tm += dt
        value = upd / tm
        sample = (f"per step {per} consecutive gates of one Trotter step of the same chain at n=26 (1 GiB "
                  f"complex128), {cores} threads")
        ms = tm / args.steps * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm, state vector (default)
def run_ours_sv(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build
    from paper_2401_06861_gb300.sim import Plan, State, launch_count

    build.build()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    n = SV_N
    gates, h, zt, ht = sv_workload()
    zzt = [t for t in ht if t[0] == 0]
    xt = [t for t in ht if t[0] != 0]
    updates = sv_gate_updates(gates, n)
    t0 = time.perf_counter()
    plan = Plan(L.SV, n, gates, L.F64)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    st = State(L.SV, n, L.F64, stream=stream.cuda_stream)
    # NVRTC time of the plan's distinct sweep kernels (host-only compile, the
    # same compiles a cold first run makes), then the first run
    t0 = time.perf_counter()
    plan.jit_check()
    compile_s = time.perf_counter() - t0
    st.run(plan)
    st.sync()

    def step(ev=None):
        st.reset()
        if ev is not None:
            ev[0].record(stream)
        st.run(plan)
        if ev is not None:
            ev[1].record(stream)
        z = st.expect(zt)
        e = st.expect(ht, sum=True)
        return z, e

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    clocks = Clocks(dev)
    n0 = launch_count()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweep_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start.record(stream)
    for k in range(args.steps):
        z, e = step(sweep_ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - n0
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    sweep_ms = sum(a.elapsed_time(b) for a, b in sweep_ev) / args.steps
    ms = reduce_max(ms, ws)
    value = job_rate(updates, ws, ms / 1e3)
    zz = st.expect(zzt)
    x = st.expect(xt)

    # end to end through the public ABI from host buffers: the host gate list
    # in (one-shot call: lowering, table upload, run), results copied back
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st.reset()
        st.apply(gates)
        z2 = st.expect(zt)
        e2 = st.expect(ht, sum=True)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = reduce_max(e2e_s, ws)
    assert abs(e2 - e) <= 1e-12 and np.max(np.abs(z2 - z)) <= 1e-12, "e2e result differs from device-timed run"
    h2d = 56 * len(gates) + 24 * (len(zt) + len(ht))
    d2h = 8 * (len(zt) + 1)

    # roofline of the dominant kernel: arithmetic-pipe bound, HBM beside it.
    # The instructions per amplitude are counted on the generated kernels
    # (FP64 path: one FP64 instruction per multiply-add or multiply;
    # double-word path: the FP32 instructions of its operations).
    dw_ran = plan.last_run_dw()
    fmas, muls, instr, _ = plan.kernel_arith(dw=dw_ran)
    nlaunch = info["sweeps"]
    launch_s = sweep_ms / 1e3 / nlaunch
    if dw_ran:
        pipe, kname = "FP32", SV_KERNEL_DW
        peak = probe_rate(L.PROBE_FP32_FMA)
    else:
        pipe, kname = "FP64", SV_KERNEL
        peak = probe_rate(L.PROBE_FP64_FMA)
    achieved = instr * 2.0 ** n / (sweep_ms / 1e3)
    hbm = info["bytes"] / (sweep_ms / 1e3) / 1e9
    traffic = traffic_per_launch(SV_TRAFFIC_FILE_DW if dw_ran else SV_TRAFFIC_FILE, JIT_SRCS)
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                "unit": f"{pipe} Ginstr/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"measured in this run (nwq_peak_probe: {pipe} FMA chains on every SM)",
                "kernel": kname, f"{pipe.lower()}_instr_per_amplitude": instr,
                "launches_per_step": nlaunch, "ms_per_launch": launch_s * 1e3,
                "algorithmic_bytes_per_launch": info["bytes"] / nlaunch, "hbm_gbs": hbm,
                "hbm_frac": hbm / _peaks()["hbm_gbs"],
                "note": "timed per plan run (the sweeps" + ("; the state keeps the double-word layout from step to "
                                                            "step: the reset writes |0..0> in it and the expectation "
                                                            "passes read it, so no layout conversion runs"
                                                            if dw_ran else "") + ")"}

    # the same circuit on the FP64 pipe (one plan run), beside the default path
    fp64_side = None
    if dw_ran and not args.no_fp64_side:
        with Plan(L.SV, n, gates, L.F64, flags=L.PLAN_FP64) as p64:
            st.reset()
            st.run(p64)  # compiles its kernels
            st.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st.run(p64)
            b.record(stream)
            torch.cuda.synchronize()
            z64 = st.expect(zt)
            e64 = st.expect(ht, sum=True)
        t64 = a.elapsed_time(b) / 1e3
        fp64_side = {"plan_run_s": t64, "double_word_plan_run_s": sweep_ms / 1e3, "speedup": t64 / (sweep_ms / 1e3),
                     "max_z_diff": float(np.max(np.abs(z64 - z))), "energy_diff": abs(e64 - e)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = sv_cpu_baseline()
        cpu["oracle_check"] = sv_oracle_check(gates, h, z, zz, x, e)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32x2" if dw_ran else "f64", "data": "synthetic",
                "config": config_of("sv", ws),
                "arithmetic": ("double-word: each FP64 value as two floats (about 48 significant bits), FP32 pipe; "
                               "complex128 storage between plan runs; FP64 parity tolerance 1e-12") if dw_ran
                else "FP64",
                "plan": {"form": "fused (reusable)" + (", double-word" if dw_ran else ""), "sweeps": info["sweeps"],
                         "operators": info["ops"], "create_s": plan_s},
                "gates_per_s": job_rate(len(gates), ws, ms / 1e3),
                "e2e": {"value": job_rate(updates, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                        "path": "nwq_sv_apply_circuit from the host gate list, then nwq_expect_pauli_sum",
                        "cold_compile_s": compile_s,
                        "note": "the one-shot calls find the specialised kernels compiled by the timed plan; "
                                "a cold process would first spend cold_compile_s in NVRTC (the plan's distinct "
                                "sweep kernels, compiled on the host)"},
                "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": ck,
                "step_split_ms": {"plan_run": sweep_ms, "reset_and_expectations": ms - sweep_ms},
                "fp64_pipe_path": fp64_side,
                "results": {"energy": e, "z0": float(z[0]), "norm": st.norm()}}
        print(json.dumps(line), flush=True)
    st.close()
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- GPU arm, density matrix
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build
    from paper_2401_06861_gb300.sim import Plan, State, launch_count

    build.build()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    gates, noise, zt, ht = workload()
    plan = Plan(L.DM, N, gates, L.F64, noise)
    info = plan.info()
    st = State(L.DM, N, L.F64, stream=stream.cuda_stream)
    ro = noise["readout_e"]
    gate_updates = len(gates) * 4.0 ** N

    def step(ev=None):
        st.reset()
        if ev is not None:
            ev[0].record(stream)
        st.run(plan)
        if ev is not None:
            ev[1].record(stream)
        z = st.expect(zt)
        e = st.expect(ht, sum=True)
        p = st.probs(ro)
        return z, e, p

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    clocks = Clocks(dev)
    n0 = launch_count()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweep_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start.record(stream)
    for k in range(args.steps):
        z, e, p = step(sweep_ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - n0
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    sweep_ms = sum(a.elapsed_time(b) for a, b in sweep_ev) / args.steps
    ms = reduce_max(ms, ws)
    value = job_rate(gate_updates, ws, ms / 1e3)

    # end to end through the public ABI with host buffers: host circuit in,
    # plan built and uploaded, run, results copied back, every step
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.reset()
        st.apply(gates, noise)
        z2 = st.expect(zt)
        e2 = st.expect(ht, sum=True)
        p2 = st.probs(ro)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = reduce_max(e2e_s, ws)
    assert abs(e2 - e) <= 1e-12 and np.max(np.abs(p2 - p)) <= 1e-15, "e2e result differs from device-timed run"
    h2d = info["table_bytes"] + 24 * (len(zt) + len(ht))
    d2h = 8 * (len(zt) + 1 + (1 << N))

    # roofline of the dominant kernel (the DM sweep), from the live events;
    # multiply-adds per element counted on the generated kernels
    dw_ran = plan.last_run_dw()
    fmas, muls, per_elem, _ = (plan.kernel_arith(dw=dw_ran) if JIT
                               else (info["fma_per_elem"], 0.0, info["fma_per_elem"], 0))
    nlaunch = info["sweeps"]
    launch_s = sweep_ms / 1e3 / nlaunch
    if dw_ran:  # FP32 instructions of the double-word kernels against the FP32 pipe
        instr = per_elem * 4.0 ** N / nlaunch
        achieved = instr / launch_s / 1e9
        peak = probe_rate(L.PROBE_FP32_FMA) / 1e9
        unit, pipe, kname = "FP32 Ginstr/s", "FP32", KERNEL_NAME_DW
    else:  # FP64 flops (2 per multiply-add) against the FP64 pipe
        achieved = 2.0 * (fmas + muls) * 4.0 ** N / nlaunch / launch_s / 1e12
        peak = 2.0 * probe_rate(L.PROBE_FP64_FMA) / 1e12
        unit, pipe, kname = "TFLOP/s", "FP64", KERNEL_NAME
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak,
                "traffic": traffic_per_launch(TRAFFIC_FILE_DW if dw_ran else TRAFFIC_FILE, KERNEL_SRCS),
                "peak_source": f"measured in this run (nwq_peak_probe: {pipe} FMA chains on every SM)",
                "kernel": kname, "fma_per_element": fmas,
                "launches_per_step": nlaunch, "ms_per_launch": launch_s * 1e3,
                "algorithmic_bytes_per_launch": info["bytes"] / nlaunch,
                "hbm_gbs": info["bytes"] / nlaunch / launch_s / 1e9,
                "hbm_frac": info["bytes"] / nlaunch / launch_s / 1e9 / _peaks()["hbm_gbs"]}

    fp64_side = None
    if dw_ran and not args.no_fp64_side:
        with Plan(L.DM, N, gates, L.F64, noise, flags=L.PLAN_FP64) as p64:
            st.reset()
            st.run(p64)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                st.reset()
                st.run(p64)
            b.record(stream)
            torch.cuda.synchronize()
            e64 = st.expect(ht, sum=True)
        t64 = a.elapsed_time(b) / args.steps / 1e3
        fp64_side = {"reset_and_plan_run_s": t64, "double_word_plan_run_s": sweep_ms / 1e3,
                     "speedup": t64 / (sweep_ms / 1e3), "energy_diff": abs(e64 - e)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, dt = oracle_sample(gates, noise, 1)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"first noisy gate (CX(0,1) + depolarising + relaxation) of the n={N} circuit "
                         f"from |0><0|, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32x2" if dw_ran else "f64", "data": "synthetic",
                "config": config_of("dm", ws),
                "arithmetic": ("double-word: each FP64 value as two floats (about 48 significant bits), FP32 pipe; "
                               "FP64 storage between plan runs; FP64 parity tolerance 1e-12") if dw_ran else "FP64",
                "plan": {"sweeps": info["sweeps"], "operators": info["ops"]},
                "e2e": {"value": job_rate(gate_updates, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": ck,
                "fp64_pipe_path": fp64_side,
                "results": {"energy": e, "z0": float(z[0]), "prob_sum": float(p.sum())}}
        print(json.dumps(line), flush=True)
    st.close()
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other workloads
# These print one JSON line each for the design notes; the default run above
# is the headline measurement.


def run_sv_cases(args):
    """Large state vector: TFIM depth 10 with random h_i, fused sweeps vs one
    gate per pass, FP32 and FP64; gate-updates/s and HBM GB/s."""
    import numpy as np
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, inputs
    from paper_2401_06861_gb300.sim import Plan, State
    build.build()
    stream = torch.cuda.current_stream()
    peak = _peaks()["hbm_gbs"]
    all_cases = {"fused32": (args.sv_n, L.F32, 0, args.steps),
                 "fused64": (args.sv_n - 1, L.F64, 0, max(1, args.steps // 3)),
                 "plain32": (args.sv_n, L.F32, L.PLAN_PLAIN, 1),
                 "tc32": (args.sv_n, L.F32, L.PLAN_TC, max(1, args.steps // 3)),
                 "commute32": (args.sv_n, L.F32, L.PLAN_COMMUTE, args.steps),
                 "nocommute32": (args.sv_n, L.F32, L.PLAN_NO_COMMUTE, args.steps)}
    cases = [all_cases[c] for c in args.sv_cases.split(",")]
    for n, dtype, flags, steps in cases:
        if args.sv_circuit == "tfim":
            gates, h = inputs.large_sv_tfim(n, steps=args.sv_depth)
            wname = f"sv_tfim_n{n}_depth{args.sv_depth}"
        else:  # generic dense one- and two-qubit gates on random qubits (half two-qubit)
            ng = 10 * n
            gates = inputs.random_circuit(n, ng, 2401 + n, names=["MAT1", "MAT2"], two_qubit_frac=0.5)
            h = np.ones(n)
            wname = f"sv_random2q_n{n}_{ng}gates"
        plan = Plan(L.SV, n, gates, dtype, None, flags)
        info = plan.info()
        st = State(L.SV, n, dtype, stream=stream.cuda_stream)
        st.run(plan)
        st.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            st.reset()
            a.record(stream)
            st.run(plan)
            b.record(stream)
        torch.cuda.synchronize()
        sec = sum(a.elapsed_time(b) for a, b in ev) / steps / 1e3
        e = st.expect(inputs.tfim_terms(n, 1.0, h), sum=True, normalize=True)
        nrm = st.norm()
        st.close()
        gb = info["bytes"] / sec / 1e9
        if flags & L.PLAN_TC:  # dense blocks on the tensor cores: HBM bound, TF32 pipe reported beside it
            tf = 2.0 * info["fma_per_elem"] * 2.0 ** n / sec / 1e12
            tf_peak = _peaks().get("bf16_tflops", 1900.0) * 1.1 / 2.25  # TF32 = measured bf16 x nominal TF32/bf16 ratio
            roof = {"bound": "hbm", "achieved": gb, "peak": peak, "unit": "GB/s", "frac": gb / peak,
                    "tf32_tflops": tf, "tf32_peak": tf_peak, "tf32_frac": tf / tf_peak}
        elif dtype == L.F32:  # complex64: HBM bound
            roof = {"bound": "hbm", "achieved": gb, "peak": peak, "unit": "GB/s", "frac": gb / peak,
                    "fp_ops_per_amp": info["fma_per_elem"]}
        else:  # complex128: arithmetic-pipe bound (double words: FP32 pipe; else FP64), instructions as generated
            dw_ran = plan.last_run_dw()
            _, _, instr, _ = plan.kernel_arith(dw=dw_ran)
            pipe = "FP32" if dw_ran else "FP64"
            rate = probe_rate(L.PROBE_FP32_FMA if dw_ran else L.PROBE_FP64_FMA)
            ach = instr * 2.0 ** n / sec
            roof = {"bound": "alu", "achieved": ach, "peak": rate, "unit": f"{pipe} instructions/s",
                    "frac": ach / rate, "instr_per_amp": instr, "hbm_gbs": gb, "hbm_frac": gb / peak}
        plan.close()
        pname = ("tc" if flags & L.PLAN_TC else "fused_no_commute" if flags & L.PLAN_NO_COMMUTE
                 else "fused_commute" if flags & L.PLAN_COMMUTE
                 else "plain" if flags else "fused")
        line = {"workload": wname, "plan": pname,
                "dtype": "c64" if dtype == L.F32 else "c128", "metric": "gate-updates/s",
                "value": len(gates) * 2.0 ** n / sec, "unit": "gate-updates/s", "s_per_circuit": sec,
                "sweeps": info["sweeps"], "operators": info["ops"], "roofline": roof, "energy": e, "norm": nrm}
        print(json.dumps(line), flush=True)
        torch.cuda.empty_cache()


def run_sv_errors(args):
    """Large state vector, errors measured against the FP64 path: the depth-10
    TFIM chain at n = sv_n - 1 (33: a 128 GiB complex128 state and a 64 GiB
    complex64 state fit together) run in complex128 (fused), then in complex64
    with each plan (fused sweeps, one gate per pass, tensor-core blocks); per
    plan the max absolute amplitude error over all 2^n amplitudes and the
    relative energy error against the complex128 state."""
    import numpy as np  # noqa: F401
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, inputs
    from paper_2401_06861_gb300.sim import Plan, State
    build.build()
    n = args.sv_n - 1
    gates, h = inputs.large_sv_tfim(n, steps=args.sv_depth)
    terms = inputs.tfim_terms(n, 1.0, h)
    hnorm = float(sum(abs(t[2]) for t in terms))
    ref = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    with State(L.SV, n, L.F64, buf=ref.data_ptr(), buf_bytes=ref.numel() * 16) as st, Plan(L.SV, n, gates, L.F64) as p:
        st.run(p)
        e_ref = st.expect(terms, sum=True)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    chunk = 1 << 27
    for name, flags in (("fused", 0), ("plain", L.PLAN_PLAIN), ("tc", L.PLAN_TC)):
        with State(L.SV, n, L.F32, buf=psi.data_ptr(), buf_bytes=psi.numel() * 8) as st, \
                Plan(L.SV, n, gates, L.F32, flags=flags) as p:
            st.run(p)
            e = st.expect(terms, sum=True, normalize=True)
            nrm = st.norm()
        torch.cuda.synchronize()
        err = 0.0
        for a in range(0, 1 << n, chunk):
            d = (psi[a:a + chunk].to(torch.complex128) - ref[a:a + chunk]).abs().max().item()
            err = max(err, d)
        line = {"workload": f"sv_tfim_n{n}_depth{args.sv_depth}_errors_vs_fp64", "plan": name, "dtype": "c64",
                "reference": "the same circuit in complex128 (fused plan)", "max_abs_amplitude_error": err,
                "rel_energy_error": abs(e - e_ref) / max(abs(e_ref), hnorm), "energy": e, "energy_fp64": e_ref,
                "norm": nrm, "tolerance": {"amplitude": 1e-5, "rel_energy": 1e-6}}
        print(json.dumps(line), flush=True)
    del ref, psi
    torch.cuda.empty_cache()


def run_vqe(args):
    """Batched VQE energies: n = 12 hardware-efficient ansatz (4 layers, 96
    parameters), 4096 sets, energies for h in {0.5, 1, 2}; batched FP32 and
    FP64 (double words, and the FP64 pipe) vs the per-circuit plain FP64 path."""
    import numpy as np
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, inputs
    from paper_2401_06861_gb300.sim import Batch, State
    build.build()
    n, layers, nsets = 12, 4, 4096
    hs = (0.5, 1.0, 2.0)
    gates, pidx = inputs.hea_ansatz(n, layers)
    params = inputs.hea_params(n, layers, nsets, seed=4096)
    terms = inputs.zz_terms(n) + inputs.x_terms(n)
    coeffs = np.array([[-1.0] * (n - 1) + [-h] * n for h in hs])
    stream = torch.cuda.current_stream()
    p = torch.from_numpy(params).cuda()
    res = {}
    # FP64 batches run in double words by default; the FP64-pipe kernel is timed beside them
    for dtype, pipe, name in ((L.F32, False, "f32"), (L.F64, False, "f64"), (L.F64, True, "f64_fp64_pipe")):
        b = Batch([dict(n=n, gates=gates, param_index=pidx, terms=terms, coeffs=coeffs)], layers * 2 * n, dtype,
                  stream=stream.cuda_stream)
        out = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
        if not pipe:
            shape = b.autotune(p.data_ptr(), nsets, out.data_ptr(), reps=3, stream=stream.cuda_stream)
        else:  # the autotuner times the default arithmetic: the same search here, with the flag
            shape = None
            for fusion in (0, 1):
                for threads in (128, 256, 512):
                    b.set_shape(threads, fusion)
                    b.run(p.data_ptr(), nsets, out.data_ptr(), stream=stream.cuda_stream, fp64_pipe=True)
                    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    t0.record(stream)
                    for _ in range(3):
                        b.run(p.data_ptr(), nsets, out.data_ptr(), stream=stream.cuda_stream, fp64_pipe=True)
                    t1.record(stream)
                    torch.cuda.synchronize()
                    ms = t0.elapsed_time(t1) / 3
                    if shape is None or ms < shape["ms"]:
                        shape = dict(threads=threads, fusion=fusion, ms=ms)
            b.set_shape(shape["threads"], shape["fusion"])
        for _ in range(3):
            b.run(p.data_ptr(), nsets, out.data_ptr(), stream=stream.cuda_stream, graph=True, fp64_pipe=pipe)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            b.run(p.data_ptr(), nsets, out.data_ptr(), stream=stream.cuda_stream, graph=True, fp64_pipe=pipe)
        t1.record(stream)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / args.steps / 1e3
        res[name] = (out.cpu().numpy(), sec, shape)
        b.close()
    # per-circuit plain FP64 path on a sample of the sets
    sample = 64
    t0 = time.perf_counter()
    plain = []
    for s in range(sample):
        g = [(name, q, (params[s][k],) if k >= 0 else prm) for (name, q, prm), k in zip(gates, pidx)]
        with State(L.SV, n, L.F64, stream=stream.cuda_stream) as st:
            st.apply(g, flags=L.PLAN_PLAIN)
            plain.append([st.expect(inputs.tfim_terms(n, 1.0, h), sum=True) for h in hs])
    psec = (time.perf_counter() - t0) / sample
    plain = np.array(plain)
    ref = res["f64"][0]
    norm1 = np.array([(n - 1) + n * h for h in hs])
    for name in ("f32", "f64", "f64_fp64_pipe"):
        out, sec, shape = res[name]
        err = float(np.max(np.abs(out - ref) / np.maximum(np.abs(ref), norm1)))
        line = {"workload": "vqe_hea_n12_4layers_4096sets", "path": f"batched_{name}", "metric": "energies/s",
                "value": 3 * nsets / sec, "unit": "energies/s", "ms_per_batch": sec * 1e3,
                "rel_energy_err_vs_batched_f64": err,
                "vs_plain_f64_per_circuit": (3 * nsets / sec) / (3 / psec),
                "arithmetic": {"f32": "FP32", "f64": "FP64 in double words (FP32 pipe)",
                               "f64_fp64_pipe": "FP64 pipe"}[name],
                "kernel_shape": {"threads": shape["threads"], "gate_fusion": shape["fusion"], "autotuned": True}}
        print(json.dumps(line), flush=True)
    err = float(np.max(np.abs(plain - ref[:sample]) / np.maximum(np.abs(ref[:sample]), norm1)))
    print(json.dumps({"workload": "vqe_hea_n12_4layers_4096sets", "path": "plain_f64_per_circuit",
                      "metric": "energies/s", "value": 3 / psec, "unit": "energies/s",
                      "sample": f"{sample} sets, host wall clock", "rel_energy_err_vs_batched_f64": err}), flush=True)


def run_dm32(args):
    """The headline noisy DM TFIM (n = 13, 20 steps) in FP32 storage and
    arithmetic (FP64 reductions): gate-updates/s, HBM roofline, and the energy
    against the FP64 path."""
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build
    from paper_2401_06861_gb300.sim import Plan, State
    build.build()
    stream = torch.cuda.current_stream()
    gates, noise, zt, ht = workload()
    e = {}
    for dtype in ((L.F32,) if args.f32_only else (L.F64, L.F32)):
        with Plan(L.DM, N, gates, dtype, noise) as plan, State(L.DM, N, dtype, stream=stream.cuda_stream) as st:
            info = plan.info()
            for _ in range(3):
                st.reset()
                st.run(plan)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                st.reset()
                st.run(plan)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / args.steps / 1e3
            e[dtype] = (st.expect(ht, sum=True), sec, info)
    e64 = e[L.F64][0] if L.F64 in e else float("nan")
    en, sec, info = e[L.F32]
    gb = info["bytes"] / sec / 1e9
    peak = _peaks()["hbm_gbs"]
    norm1 = sum(abs(t[2]) for t in ht)
    line = {"workload": WORKLOAD, "path": "dm_f32", "metric": METRIC, "value": len(gates) * 4.0 ** N / sec,
            "unit": UNIT, "ms_per_step": sec * 1e3, "dtype": "f32", "sweeps": info["sweeps"],
            "roofline": {"bound": "hbm", "achieved": gb, "peak": peak, "unit": "GB/s", "frac": gb / peak},
            "energy": en, "energy_f64": e64, "rel_energy_err_vs_f64": abs(en - e64) / max(abs(e64), norm1),
            "f64_ms_per_step": e[L.F64][1] * 1e3 if L.F64 in e else None}
    print(json.dumps(line), flush=True)


def run_vqe_sharded(args, ws, rank, local):
    """Batched VQE over several GPUs (torchrun): the 4096 sets split into one
    share per rank (paper_2401_06861_gb300/dispatch.py), each share one
    batched FP32 launch on that rank's GPU, energies gathered on rank 0.
    Whole-job energies/s = 3 x 4096 / the slowest rank's time (strong scaling:
    the total is fixed)."""
    import numpy as np
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, dispatch, inputs
    from paper_2401_06861_gb300.sim import Batch
    build.build()
    torch.cuda.set_device(local)
    n, layers, nsets = 12, 4, 4096
    hs = (0.5, 1.0, 2.0)
    gates, pidx = inputs.hea_ansatz(n, layers)
    params = inputs.hea_params(n, layers, nsets, seed=4096)
    terms = inputs.zz_terms(n) + inputs.x_terms(n)
    coeffs = np.array([[-1.0] * (n - 1) + [-h] * n for h in hs])
    stream = torch.cuda.current_stream()
    timing = {}

    def run_share(lo, hi, share):
        p = torch.from_numpy(np.ascontiguousarray(share)).cuda()
        out = torch.zeros(max(hi - lo, 1), 3, dtype=torch.float64, device="cuda")
        b = Batch([dict(n=n, gates=gates, param_index=pidx, terms=terms, coeffs=coeffs)], layers * 2 * n, L.F32,
                  stream=stream.cuda_stream)
        for _ in range(max(args.warmup, 3)):
            b.run(p.data_ptr(), hi - lo, out.data_ptr(), stream=stream.cuda_stream, graph=True)
        torch.cuda.synchronize()
        import torch.distributed as dist
        dist.barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            b.run(p.data_ptr(), hi - lo, out.data_ptr(), stream=stream.cuda_stream, graph=True)
        t1.record(stream)
        torch.cuda.synchronize()
        timing["s"] = t0.elapsed_time(t1) / args.steps / 1e3
        b.close()
        return out[:hi - lo].cpu().numpy()

    energies = dispatch.run_batched(run_share, params, ws, rank)
    sec = reduce_max(timing["s"], ws)
    if rank == 0:
        print(json.dumps({"workload": "vqe_hea_n12_4layers_4096sets", "path": "batched_f32_sharded",
                          "metric": "energies/s", "value": 3 * nsets / sec, "unit": "energies/s", "n_gpus": ws,
                          "scaling": "strong", "ms_per_batch": sec * 1e3, "sets_per_rank": nsets // ws,
                          "energies_shape": list(energies.shape)}), flush=True)
    import torch.distributed as dist
    dist.destroy_process_group()
    return 0


def run_serve_sharded(args, ws, rank, local):
    """Serving over several GPUs (torchrun): the request stream dealt
    round-robin to the ranks (paper_2401_06861_gb300/dispatch.py), each rank
    serving its share with its own executor, streams and 150 GB budget;
    results gathered on rank 0."""
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, dispatch, inputs
    from paper_2401_06861_gb300.serve import GpuExecutor, Server, summarize
    build.build()
    torch.cuda.set_device(local)
    reqs = inputs.serve_requests(rate=200.0, duration=args.serve_seconds, seed=200)
    warm = inputs.serve_requests(rate=200.0, duration=1.0, seed=7, sv_n=(8, 20), dm_n=(6, 9))
    Server(GpuExecutor(L.F32), slots=8, dtype=L.F32).serve(warm)
    import torch.distributed as dist
    dist.barrier()
    res, stats = dispatch.serve_sharded(
        lambda: Server(GpuExecutor(L.F32), slots=args.serve_slots, dtype=L.F32, budget_bytes=150e9), reqs, ws, rank)
    if rank == 0:
        wall = max(st["wall"] for st in stats)
        s = summarize(res, wall)
        s.update(workload=f"serve_poisson200_{args.serve_seconds:g}s", path="served_f32_sharded", n_gpus=ws,
                 metric="circuits/s", value=s["circuits_per_s"], unit="circuits/s", per_rank=stats)
        print(json.dumps(s), flush=True)
    dist.destroy_process_group()
    return 0


def run_vqe_cobyla(args):
    """VQE outer loop (COBYLA) on the Ising chain: noise-free n = 12 (4 layers,
    96 parameters; 256 batched starts, then COBYLA with one launch per energy)
    and noisy n = 6 (density matrix with the device noise model, 3 layers)."""
    import numpy as np

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, inputs, vqe
    build.build()
    cases = [("noise_free", 12, 4, None, L.F64, 256), ("noisy", 6, 3, inputs.noise_params(6, seed=2401), L.F64, 1)]
    for name, n, layers, noise, dtype, starts in cases:
        ef = vqe.NoiseFreeEnergy(n, layers, dtype=dtype) if noise is None else vqe.NoisyEnergy(n, layers, noise, dtype)
        t0 = time.perf_counter()
        r = vqe.minimize(ef, ef.nparams, starts=starts, batch_energy=getattr(ef, "batch", None),
                         maxiter=args.vqe_maxiter, tol=1e-6)
        sec = time.perf_counter() - t0
        line = {"workload": f"vqe_cobyla_{name}_n{n}_{layers}layers", "metric": "energies/s",
                "value": ef.nevals / sec, "unit": "energies/s", "wall_s": sec, "evaluations": ef.nevals,
                "cobyla_nfev": r["nfev"], "energy": r["energy"], "dtype": "f64",
                "note": "host wall clock of the whole optimisation (scipy COBYLA + one library call per energy)"}
        print(json.dumps(line), flush=True)
        ef.close()


def run_traj(args):
    """Noisy TFIM n = 12 (20 Trotter steps, device noise model) two ways: the
    density matrix (4^12 FP64 Pauli coefficients) and 4096 quantum
    trajectories (state vectors in shared memory); <H> and time of each."""
    import numpy as np
    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, inputs, sim
    build.build()
    n, steps, ntraj = 12, 20, 4096
    gates, noise = inputs.dm_noisy_tfim(n, steps)
    terms = inputs.tfim_terms(n)
    coeffs = [[t[2] for t in terms]]
    with sim.State(L.DM, n, L.F64) as st, sim.Plan(L.DM, n, gates, L.F64, noise) as plan:
        st.run(plan)
        st.sync()
        t0 = time.perf_counter()
        st.reset()
        st.run(plan)
        e_dm = st.expect(terms, sum=True)
        dm_s = time.perf_counter() - t0
    # F64 trajectories run in double words by default; NWQ_DW=0 gives the FP64-pipe kernel
    for dtype, name, env_dw in ((L.F64, "f64", None), (L.F64, "f64_fp64_pipe", "0"), (L.F32, "f32", None)):
        if env_dw is None:
            os.environ.pop("NWQ_DW", None)
        else:
            os.environ["NWQ_DW"] = env_dw
        sim.trajectories(n, gates, noise, terms, coeffs, 64, dtype, seed=1)  # warm-up
        d = sim.trajectory_draws(n, gates, noise)
        u = np.random.default_rng(2).random((ntraj, d))
        t0 = time.perf_counter()
        e = sim.trajectories(n, gates, noise, terms, coeffs, ntraj, dtype, uniforms=u)[:, 0]
        sec = time.perf_counter() - t0
        line = {"workload": f"noisy_tfim_n{n}_{steps}steps_trajectories", "path": f"trajectories_{name}",
                "metric": "trajectories/s", "value": ntraj / sec, "unit": "trajectories/s", "trajectories": ntraj,
                "draws_per_trajectory": d, "wall_s": sec, "energy_mean": float(e.mean()),
                "energy_stderr": float(e.std() / np.sqrt(ntraj)), "energy_density_matrix": e_dm,
                "density_matrix_s": dm_s,
                "arithmetic": {"f64": "FP64 in double words (FP32 pipe)", "f64_fp64_pipe": "FP64 pipe",
                               "f32": "FP32"}[name],
                "note": "host wall clock incl. the host->device copy of the draws; the density matrix value is one "
                        "FP64 run of the same circuit"}
        print(json.dumps(line), flush=True)
    os.environ.pop("NWQ_DW", None)


def run_peaks(args):
    """The arithmetic roofline denominators: nwq_peak_probe (independent FMA
    chains on every SM, about 60 ms per call after a warm-up launch) for the
    FP64 and FP32 pipes, five calls each with nvidia-smi clocks sampled
    around them; one JSON line per pipe."""
    import statistics

    import torch

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build
    build.build()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for what, pipe in ((L.PROBE_FP64_FMA, "FP64"), (L.PROBE_FP32_FMA, "FP32")):
        probe_rate(what)  # warm-up
        clocks = Clocks(dev)
        vals = [probe_rate(what) for _ in range(5)]
        ck = clocks.stop()
        med = statistics.median(vals)
        mhz = (ck or {}).get("sm_mhz") or 0.0
        print(json.dumps({"workload": "peak_probe", "pipe": pipe, "metric": "FMA instructions/s", "value": med,
                          "unit": "FMA/s", "flops": 2 * med, "calls": vals, "sms": sms,
                          "fma_per_sm_per_clock": med / (sms * mhz * 1e6) if mhz else None, "clocks": ck,
                          "kernel": "fma_chains (csrc/probe.cu): " + ("8 FP64 chains, 4096 iterations per thread"
                                                                      if what == L.PROBE_FP64_FMA else
                                                                      "16 FP32 chains, 2^17 iterations per thread")}),
              flush=True)


def serve_oracle_check(reqs, res, budget_s=20.0, every=100):
    """cpu_baseline leg of the serving line: the CPU oracle on a sample of the
    served requests (every 100th completed request with SV n <= 16 or DM n <= 9,
    until about 20 s of CPU work), timed, and the largest error of the served
    FP32 results against it."""
    import numpy as np

    import oracle
    oracle.lib()
    byid = {q["id"]: q for q in reqs}
    cand = [i for i in sorted(res) if res[i]["error"] is None and
            ((byid[i]["kind"] == "sv" and byid[i]["n"] <= 16) or (byid[i]["kind"] == "dm" and byid[i]["n"] <= 9))]
    zerr = eerr = 0.0
    done = 0
    t0 = time.perf_counter()
    for i in cand[::every]:
        q, n = byid[i], byid[i]["n"]
        if q["kind"] == "sv":
            psi = oracle.sv_run(n, q["gates"])
            z, ev = oracle.sv_expect(psi, n, q["z_terms"]), oracle.sv_expect(psi, n, q["h_terms"])
        else:
            rho = oracle.dm_run(n, q["gates"], q["noise"])
            z, ev = oracle.dm_expect(rho, n, q["z_terms"]), oracle.dm_expect(rho, n, q["h_terms"])
        e = oracle.energy(ev, q["h_terms"])
        norm1 = sum(abs(t[2]) for t in q["h_terms"])
        zerr = max(zerr, float(np.max(np.abs(np.asarray(res[i]["z"]) - np.asarray(z)))))
        eerr = max(eerr, abs(res[i]["energy"] - e) / max(abs(e), norm1))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    sec = time.perf_counter() - t0
    check = {"requests": done, "max_z_err": zerr, "max_rel_energy_err": eerr,
             "tolerance": {"z": 1e-5, "rel_energy": 1e-6}}
    base = {"value": done / sec if sec > 0 else 0.0, "unit": "circuits/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{done} served requests (every {every}th completed with SV n<=16 or DM n<=9), {sec:.1f} s"}
    return check, base


def run_serve(args):
    """Serving: Poisson stream (200 circuits/s for --serve-seconds), 70% SV
    n ~ U{8..26}, 30% DM n ~ U{6..12}; served FP32 (continuous batching,
    8 streams) vs plain FP64 serial on the first seconds of the same stream."""
    import numpy as np

    from paper_2401_06861_gb300 import _lib as L
    from paper_2401_06861_gb300 import build, inputs
    from paper_2401_06861_gb300.serve import GpuExecutor, Server, summarize
    build.build()
    reqs = inputs.serve_requests(rate=200.0, duration=args.serve_seconds, seed=200)
    warm = inputs.serve_requests(rate=200.0, duration=1.0, seed=7, sv_n=(8, 20), dm_n=(6, 9))
    Server(GpuExecutor(L.F32), slots=8, dtype=L.F32).serve(warm)
    ex = GpuExecutor(L.F32)
    srv = Server(ex, slots=args.serve_slots, dtype=L.F32, budget_bytes=150e9)
    res = srv.serve(reqs)
    s = summarize(res, srv.wall)
    errs = {}
    for r in res.values():
        if r["error"]:
            errs[r["error"][:120]] = errs.get(r["error"][:120], 0) + 1
    s["errors"] = errs
    s["plan_cache"] = {"hits": ex.hits, "misses": ex.misses}
    if not args.no_cpu_baseline:
        s["oracle_check"], s["cpu_baseline"] = serve_oracle_check(reqs, res)
    s["slots"] = args.serve_slots
    s.update(workload=f"serve_poisson200_{args.serve_seconds:g}s", path="served_f32", metric="circuits/s",
             value=s["circuits_per_s"], unit="circuits/s", offered=len(reqs) / args.serve_seconds,
             peak_budget_bytes=srv.ledger.peak,
             batched=sum(1 for r in res.values() if r["path"] == "batch"))
    print(json.dumps(s), flush=True)
    window = min(args.serve_seconds, args.serial_seconds)
    sub = [r for r in reqs if r["arrival"] < window]
    ser = Server(GpuExecutor(L.F64, plan_flags=L.PLAN_PLAIN), slots=1, batch_max_n=0, dtype=L.F64)
    res2 = ser.serve(sub)
    s2 = summarize(res2, ser.wall)
    s2.update(workload=f"serve_poisson200_first{window:g}s", path="plain_f64_serial", metric="circuits/s",
              value=s2["circuits_per_s"], unit="circuits/s", offered=len(sub) / window)
    print(json.dumps(s2), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--f32-only", action="store_true", help="dm32: the FP32 plan only (for profiling)")
    ap.add_argument("--no-fp64-side", action="store_true",
                    help="skip the one FP64-pipe run beside a double-word headline")
    ap.add_argument("--workload", default="sv",
                    choices=["sv", "dm", "dm32", "sv-cases", "sv-errors", "vqe", "vqe-cobyla", "serve", "traj",
                             "peaks"],
                    help="sv: the default line (n=33 complex128 TFIM, depth 10); dm: noisy DM TFIM n=13; "
                         "the others print design-note lines")
    ap.add_argument("--vqe-maxiter", type=int, default=2000)
    ap.add_argument("--sv-n", type=int, default=34)
    ap.add_argument("--sv-depth", type=int, default=10)
    ap.add_argument("--sv-circuit", default="tfim", choices=["tfim", "random2q"],
                    help="large-SV circuit: TFIM Trotter chain, or random dense one/two-qubit gates")
    ap.add_argument("--sv-cases", default="fused32,fused64,plain32,tc32",
                    help="comma list of fused32, fused64, plain32, tc32 (tensor-core blocks), "
                         "commute32 (fused, diagonal operators commuting: the default), nocommute32")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serial-seconds", type=float, default=5.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc
    if args.workload == "sv":
        return run_ours_sv(args, ws, rank, local)
    if args.workload == "sv-cases":
        return run_sv_cases(args)
    if args.workload == "sv-errors":
        return run_sv_errors(args)
    if args.workload == "vqe-cobyla":
        return run_vqe_cobyla(args)
    if args.workload == "traj":
        return run_traj(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "dm32":
        return run_dm32(args)
    if args.workload == "vqe":
        return run_vqe_sharded(args, ws, rank, local) if ws > 1 else run_vqe(args)
    if args.workload == "serve":
        return run_serve_sharded(args, ws, rank, local) if ws > 1 else run_serve(args)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
