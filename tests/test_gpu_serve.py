"""Serving loop on the GPU: results against the oracle, and each result the
same alone as in the mix (continuous batching must not couple requests)."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.serve import GpuExecutor, Server, summarize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


def small_stream(seed=11):
    return inputs.serve_requests(rate=400, duration=0.25, seed=seed, sv_n=(6, 16), dm_n=(3, 6),
                                 trotter_steps=(2, 8), hea_layers=(1, 3))


def oracle_result(r):
    n = r["n"]
    if r["kind"] == "sv":
        psi = oracle.sv_run(n, r["gates"])
        nrm = np.vdot(psi, psi).real
        z = oracle.sv_expect(psi, n, r["z_terms"]) / nrm
        e = oracle.energy(oracle.sv_expect(psi, n, r["h_terms"]), r["h_terms"]) / nrm
    else:
        rho = oracle.dm_run(n, r["gates"], r["noise"])
        z = oracle.dm_expect(rho, n, r["z_terms"])
        e = oracle.energy(oracle.dm_expect(rho, n, r["h_terms"]), r["h_terms"])
    return z, e


@pytest.mark.parametrize("dtype", [L.F32, L.F64])
def test_served_results_match_oracle(dtype):
    reqs = small_stream()
    srv = Server(GpuExecutor(dtype), slots=4, batch_max_n=12, dtype=dtype)
    res = srv.serve(reqs)
    s = summarize(res, srv.wall)
    print(f"served {s}")
    assert s["failed"] == 0
    paths = {r["path"] for r in res.values()}
    assert paths == {"batch", "stream"}
    tol_z, tol_e = (1e-12, 1e-12) if dtype == L.F64 else (1e-5, 1e-6)
    for r in reqs:
        z, e = oracle_result(r)
        got = res[r["id"]]
        norm1 = sum(abs(t[2]) for t in r["h_terms"])
        assert np.max(np.abs(got["z"] - z)) <= tol_z, (r["id"], r["kind"], r["n"])
        assert abs(got["energy"] - e) / max(abs(e), norm1) <= tol_e, (r["id"], r["kind"], r["n"])


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = small_stream(seed=12)
    mix = Server(GpuExecutor(L.F32), slots=4, batch_max_n=12).serve(reqs)
    rng = np.random.default_rng(3)
    for r in rng.choice(reqs, size=12, replace=False):
        alone = Server(GpuExecutor(L.F32), slots=1, batch_max_n=12).serve([dict(r, arrival=0.0)])
        a, m = alone[r["id"]], mix[r["id"]]
        assert a["error"] is None and m["error"] is None
        norm1 = sum(abs(t[2]) for t in r["h_terms"])
        assert np.max(np.abs(a["z"] - m["z"])) <= 1e-6
        assert abs(a["energy"] - m["energy"]) / norm1 <= 1e-6
