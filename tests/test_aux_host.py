"""Host-side configuration helpers (no GPU): the NWQ_PLAN environment override
of the plan form and the on-disk autotuning cache (NWQ_AUTOTUNE_CACHE)."""
import ctypes
import json
import os
import subprocess
import sys

import pytest

from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs, sim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import json
from paper_2401_06861_gb300 import _lib as L, inputs, sim
g = inputs.random_circuit(12, 30, 5, names=["H", "RX", "RZ", "CX", "CZ"])
out = {"ngates": len(g)}
for name, dt, kw in [("c64", L.F32, {}), ("c128", L.F64, {}), ("c64_plain_flag", L.F32, {"flags": L.PLAN_PLAIN}),
                     ("c64_tuned", L.F32, {"tuning": {"fusion_bits": 4}})]:
    with sim.Plan(L.SV, 12, g, dt, **kw) as p:
        try:
            p.tc_blocks()
            tc = True
        except L.NwqError:
            tc = False
        out[name] = {"sweeps": p.info()["sweeps"], "tc": tc}
print(json.dumps(out))
"""


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2401_06861_gb300 import build
    build.build()


def probe(env_plan):
    env = dict(os.environ)
    env.pop("NWQ_PLAN", None)
    if env_plan is not None:
        env["NWQ_PLAN"] = env_plan
    r = subprocess.run([sys.executable, "-c", PROBE], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_nwq_plan_environment_override():
    base, plain, tc = probe(None), probe("plain"), probe("tc")
    ng = base["ngates"]
    # default: fused sweeps
    assert base["c64"]["sweeps"] < ng and not base["c64"]["tc"]
    # plain: one gate per pass wherever the call names no form
    assert plain["c64"]["sweeps"] == ng and plain["c128"]["sweeps"] == ng
    assert plain["c64_tuned"]["sweeps"] == base["c64_tuned"]["sweeps"]  # an explicit tuning wins
    # tc: tensor-core blocks where supported (complex64), the default elsewhere
    assert tc["c64"]["tc"] and not tc["c128"]["tc"] and tc["c128"]["sweeps"] == base["c128"]["sweeps"]
    assert tc["c64_plain_flag"]["sweeps"] == ng and not tc["c64_plain_flag"]["tc"]  # an explicit flag wins
    assert probe("fused") == base
    commute = probe("commute")  # the default for state vectors
    assert commute["c64"]["sweeps"] == base["c64"]["sweeps"] and not commute["c64"]["tc"]
    nocommute = probe("nocommute")  # the random circuit has diagonal gates to commute
    assert nocommute["c64"]["sweeps"] >= base["c64"]["sweeps"] and not nocommute["c64"]["tc"]


class _StubLib:
    """Stands in for the library's autotuner: records calls, returns two shapes."""

    def __init__(self):
        self.calls = 0

    def nwq_plan_autotune(self, h, arr, ng, nm, flags, reps, best, bms, tried, tms, maxn, nt):
        self.calls += 1
        best._obj.tile_bits, best._obj.fusion_bits, best._obj.register_bits = 12, 4, 4
        bms._obj.value = 1.5
        tried[0].tile_bits, tried[0].fusion_bits, tried[0].register_bits = 12, 4, 4
        tried[1].tile_bits, tried[1].fusion_bits, tried[1].register_bits = 0, 5, 0
        tms[0], tms[1] = 1.5, 2.5
        nt._obj.value = 2
        return 0


class _StubState:
    kind, n, dtype, h = L.SV, 14, L.F32, ctypes.c_void_p()


def test_autotune_cache_hits_skip_the_tuner(tmp_path, monkeypatch):
    stub = _StubLib()
    monkeypatch.setattr(sim.L, "lib", lambda: stub)
    path = str(tmp_path / "tune.json")
    gates = inputs.random_circuit(14, 40, 9, names=["H", "RX", "CX"])
    r1 = sim.autotune(_StubState(), gates, cache=path)
    assert stub.calls == 1 and not r1["cached"] and r1["best"] == {"tile_bits": 12, "fusion_bits": 4,
                                                                   "register_bits": 4}
    r2 = sim.autotune(_StubState(), gates, cache=path)
    assert stub.calls == 1 and r2["cached"] and r2["best"] == r1["best"] and r2["best_ms"] == 1.5
    assert [list(t) for t in r2["tried"]] == [list(t) for t in r1["tried"]]
    # angles do not change the key; qubits and precision do
    other_angles = [(g[0], g[1], tuple(p + 0.1 for p in g[2])) for g in gates]
    assert sim.autotune(_StubState(), other_angles, cache=path)["cached"]
    moved = [(g[0], tuple((q + 1) % 14 for q in g[1]), g[2]) for g in gates]
    assert not sim.autotune(_StubState(), moved, cache=path)["cached"] and stub.calls == 2
    assert len(json.load(open(path))) == 2
    # the environment variable names the default cache file
    monkeypatch.setenv("NWQ_AUTOTUNE_CACHE", path)
    assert sim.autotune(_StubState(), gates)["cached"] and stub.calls == 2


def test_autotune_key_fields():
    g = [("H", (0,), ()), ("CX", (0, 1), ())]
    k = sim.autotune_key(L.SV, 12, L.F32, g, device="gpu-a")
    assert k == sim.autotune_key(L.SV, 12, L.F32, [("H", (0,), ()), ("CX", (0, 1), ())], device="gpu-a")
    assert k != sim.autotune_key(L.SV, 12, L.F64, g, device="gpu-a")
    assert k != sim.autotune_key(L.SV, 13, L.F32, g, device="gpu-a")
    assert k != sim.autotune_key(L.SV, 12, L.F32, g, device="gpu-b")
    assert k != sim.autotune_key(L.SV, 12, L.F32, g, flags=L.PLAN_PLAIN, device="gpu-a")
    assert k != sim.autotune_key(L.SV, 12, L.F32, [("CX", (0, 1), ()), ("H", (0,), ())], device="gpu-a")
