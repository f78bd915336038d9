"""Host-side checks of the CUDA library (no GPU needed): it loads, exports
every symbol the header declares, validates arguments, and its planner
produces a valid schedule."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2401_06861_gb300 import build
    build.build()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "nwqgb.h")).read()
    return sorted(set(re.findall(r"\b(nwq_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    syms = header_symbols()
    assert len(syms) >= 20
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    lib = L.lib()
    for s in header_symbols():
        assert getattr(lib, s).argtypes is not None or s == "nwq_last_error", s


def test_state_bytes():
    assert sim.state_bytes(L.SV, 10, L.F64) == 16 << 10
    assert sim.state_bytes(L.SV, 34, L.F32) == 8 << 34
    assert sim.state_bytes(L.DM, 13, L.F64) == 8 << 26
    assert sim.state_bytes(L.DM, 13, L.F32) == 4 << 26
    assert sim.state_bytes(L.SV, 35, L.F64) == 0
    assert sim.state_bytes(L.DM, 17, L.F64) == 0
    assert sim.state_bytes(L.SV, 0, L.F64) == 0


def test_invalid_arguments_fail_without_device():
    h = ctypes.c_void_p()
    assert L.lib().nwq_sv_create(0, L.F64, None, 0, None, ctypes.byref(h)) == L.EINVAL
    assert L.lib().nwq_dm_create(20, L.F64, None, 0, None, ctypes.byref(h)) == L.EINVAL
    assert L.lib().nwq_sv_create(4, 7, None, 0, None, ctypes.byref(h)) == L.EINVAL
    assert b"unsupported" in L.lib().nwq_last_error()
    with pytest.raises(L.NwqError):
        sim.Plan(L.SV, 3, [inputs.gate("CX", (0, 3))])
    with pytest.raises(L.NwqError):
        sim.Plan(L.SV, 3, [inputs.gate("CX", (1, 1))])
    with pytest.raises(L.NwqError):  # noise needs a density matrix
        sim.Plan(L.SV, 3, [inputs.gate("X", (0,))], noise=inputs.noise_params(3))
    with pytest.raises(L.NwqError):  # noise arrays shorter than the register
        sim.Plan(L.DM, 4, [inputs.gate("X", (0,))], noise=inputs.noise_params(3))


def _check_schedule(n, gates, kind, dtype, flags=0, noise=None):
    p = sim.Plan(kind, n, gates, dtype, noise, flags)
    sweeps, g0, ng = p.layout()
    info = p.info()
    assert sum(sweeps) == info["ops"] == len(g0)
    # every gate folded into exactly one operator, in contiguous runs
    covered = sorted((a, a + b) for a, b in zip(g0, ng))
    pos = 0
    for a, b in covered:
        assert a == pos
        pos = b
    assert pos == len(gates)
    # operators that share a qubit keep the gate order
    qs = [set(gates[a][1]).union(*[set(gates[k][1]) for k in range(a, a + b)]) for a, b in zip(g0, ng)]
    for i in range(len(g0)):
        for j in range(i + 1, len(g0)):
            if qs[i] & qs[j]:
                assert g0[i] < g0[j]
    return info


@pytest.mark.parametrize("kind,dtype", [(L.SV, L.F64), (L.SV, L.F32), (L.DM, L.F64), (L.DM, L.F32)])
@pytest.mark.parametrize("flags", [0, L.PLAN_PLAIN, L.PLAN_NO_MERGE])
def test_planner_schedule_is_a_valid_reordering(kind, dtype, flags):
    n = 9 if kind == L.SV else 6
    gates = inputs.random_circuit(n, 300, 17)
    noise = inputs.noise_params(n) if kind == L.DM else None
    info = _check_schedule(n, gates, kind, dtype, flags, noise)
    if flags == L.PLAN_PLAIN:
        assert info["sweeps"] == len(gates)


def test_planner_tfim_sweep_counts():
    # n=13 noisy DM TFIM: 20 steps x (12 merged bond blocks + 13 RX) operators
    g, noise = inputs.dm_noisy_tfim(13, 20)
    info = _check_schedule(13, g, L.DM, L.F64, 0, noise)
    assert info["ops"] == 20 * 25
    assert info["sweeps"] <= 80
    # the whole 10-qubit SV circuit fits one tile: one sweep
    info = _check_schedule(10, inputs.tfim_trotter(10), L.SV, L.F64)
    assert info["sweeps"] == 1
    # large SV: fused plan moves far fewer bytes than the gate-by-gate plan
    g, _ = inputs.large_sv_tfim(33)
    fused = sim.Plan(L.SV, 33, g, L.F32).info()
    plain = sim.Plan(L.SV, 33, g, L.F32, flags=L.PLAN_PLAIN).info()
    assert fused["bytes"] < plain["bytes"] / 20


def test_batch_create_validates_without_device():
    import ctypes
    from paper_2401_06861_gb300.sim import Batch
    g, pidx = inputs.hea_ansatz(4, 1)
    ok = dict(n=4, gates=g, param_index=pidx, terms=inputs.z_terms(4), coeffs=np.ones((1, 4)))
    for bad, msg in [(dict(ok, n=14), b"qubit count"), (dict(ok, n=2), b"qubit out of range"),
                     (dict(ok, gates=[inputs.gate("MAT2", (0, 1), np.eye(4))], param_index=[-1]), b"MAT2"),
                     (dict(ok, gates=[inputs.gate("CX", (0, 1))], param_index=[0]), b"without an angle"),
                     (dict(ok, param_index=[99] * len(g)), b"parameter index")]:
        with pytest.raises(L.NwqError) as ei:
            Batch([bad], 8, L.F64)
        assert ei.value.code == L.EINVAL
        assert msg in L.lib().nwq_last_error()


@pytest.mark.parametrize("dtype", [L.F32, L.F64])
def test_specialised_sweep_kernels_compile(dtype):
    # NVRTC needs no device: every eligible sweep's generated source must compile
    plans = [(20, inputs.large_sv_tfim(20, 3)[0], 0), (19, inputs.random_circuit(19, 400, 23), 0),
             (18, inputs.hea_ansatz(18, 3, inputs.hea_params(18, 3, 1)[0])[0], 0),
             (20, inputs.random_circuit(20, 60, 29), L.PLAN_NO_MERGE),
             (20, inputs.large_sv_tfim(20, 4)[0], L.PLAN_COMMUTE),
             (20, inputs.large_sv_tfim(20, 4)[0], L.PLAN_NO_COMMUTE)]
    total = 0
    for n, gates, flags in plans:
        p = sim.Plan(L.SV, n, gates, dtype, flags=flags)
        eligible, built = p.jit_check()
        assert built == eligible, L.lib().nwq_last_error()
        total += eligible
        p.close()
    for n in (9, 12):  # density matrices: real operators in register phases
        g, noise = inputs.dm_noisy_tfim(n, 3)
        p = sim.Plan(L.DM, n, g, dtype, noise)
        eligible, built = p.jit_check()
        assert built == eligible, L.lib().nwq_last_error()
        total += eligible
        p.close()
    assert total >= 10


def test_exit_while_kernels_compile_in_the_background():
    # a process that queues specialised-kernel compiles and exits at once must
    # exit cleanly (the compiler thread is joined before NVRTC is torn down)
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2401_06861_gb300 import _lib as L, inputs, sim\n"
        "g, noise = inputs.dm_noisy_tfim(13, 20)\n"
        "p = sim.Plan(L.DM, 13, g, L.F64, noise)\n"
        "print('pending', p.jit_prefetch())\n" % ROOT)
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
        assert "pending" in r.stdout


def test_plan_tuning_shapes_and_validation():
    g, _ = inputs.large_sv_tfim(20, 4)
    base = sim.Plan(L.SV, 20, g, L.F32).info()
    t11 = sim.Plan(L.SV, 20, g, L.F32, tuning=dict(tile_bits=11)).info()
    t13 = sim.Plan(L.SV, 20, g, L.F32, tuning=dict(tile_bits=13)).info()
    assert t11["sweeps"] >= base["sweeps"] >= t13["sweeps"]  # larger tiles, fewer passes
    f2 = sim.Plan(L.SV, 20, g, L.F32, tuning=dict(fusion_bits=2)).info()
    assert f2["ops"] >= base["ops"]  # narrower fusion, more operators
    gd, noise = inputs.dm_noisy_tfim(8, 5)
    d2 = sim.Plan(L.DM, 8, gd, L.F64, noise, tuning=dict(fusion_bits=2)).info()
    d4 = sim.Plan(L.DM, 8, gd, L.F64, noise).info()
    assert d2["ops"] > d4["ops"]  # two-qubit noisy blocks are only merged at 4 bits
    for bad, msg in [(dict(tile_bits=3), b"tile_bits"), (dict(tile_bits=16), b"tile_bits"),
                     (dict(fusion_bits=6), b"fusion_bits"), (dict(register_bits=2), b"register_bits")]:
        with pytest.raises(L.NwqError):
            sim.Plan(L.SV, 20, g, L.F32, tuning=bad)
        assert msg in L.lib().nwq_last_error()
    for rb in (3, 4):
        p = sim.Plan(L.SV, 20, g, L.F64, tuning=dict(register_bits=rb, tile_bits=12))
        e, b = p.jit_check()
        assert e == b and e > 0


def test_every_plan_passes_the_table_check():
    # the host-side check of the device tables, over many random plans and shapes
    rng = np.random.default_rng(5)
    count = 0
    for kind in (L.SV, L.DM):
        for dtype in (L.F64, L.F32):
            for n in ((3, 9, 14, 20) if kind == L.SV else (2, 5, 8, 10)):
                for flags in (0, L.PLAN_PLAIN, L.PLAN_NO_MERGE):
                    for tuning in (None, dict(tile_bits=10, fusion_bits=3, register_bits=3),
                                   dict(tile_bits=13, fusion_bits=2, register_bits=4)):
                        if tuning and (2 * (8 if dtype == L.F32 else 16) << tuning["tile_bits"]) > 200 * 1024:
                            continue
                        g = inputs.random_circuit(n, 120, int(rng.integers(1 << 30)))
                        noise = inputs.noise_params(n, seed=int(rng.integers(1 << 30))) if kind == L.DM else None
                        p = sim.Plan(kind, n, g, dtype, noise, flags, tuning=tuning)
                        p.verify()
                        p.close()
                        count += 1
    assert count >= 100


def test_table_check_is_on_with_the_environment_variable():
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2401_06861_gb300 import _lib as L, inputs, sim\n"
            "g, noise = inputs.dm_noisy_tfim(6, 3)\n"
            "sim.Plan(L.DM, 6, g, L.F64, noise)\n"
            "sim.Plan(L.SV, 12, inputs.random_circuit(12, 200, 1), L.F32)\n"
            "print('ok')\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, NWQ_CHECKS="1"))
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]


def test_complex128_x_rotations_keep_a_unit_diagonal():
    # FP64 complex plans carry the cos factor of X-rotations as a deferred
    # scalar (2 FP64 instructions per element instead of 4); long chains push
    # the scalar back into the state before its exponent leaves range
    rng = np.random.default_rng(3)
    for n in (10, 18):  # 18 qubits: large enough for the specialised kernels
        gates = []
        for i in range(900 if n == 10 else 240):
            q = int(rng.integers(n))
            gates.append(inputs.gate("RX", (q,), (float(rng.uniform(-1.5, 1.5)),)))
            if i % 3 == 2:
                gates.append(inputs.gate("CX", (q, (q + 1) % n)))
        for flags in (L.PLAN_FUSED, L.PLAN_NO_MERGE):
            f64 = sim.Plan(L.SV, n, gates, L.F64, flags=flags)
            f32 = sim.Plan(L.SV, n, gates, L.F32, flags=flags)
            f64.verify()
            e, b = f64.jit_check()
            assert e == b and (e > 0) == (n == 18), L.lib().nwq_last_error()
            assert f64.info()["fma_per_elem"] < f32.info()["fma_per_elem"]
            f64.close()
            f32.close()
    g, _ = inputs.large_sv_tfim(20, 4)
    assert sim.Plan(L.SV, 20, g, L.F64).info()["fma_per_elem"] < sim.Plan(L.SV, 20, g, L.F32).info()["fma_per_elem"]
