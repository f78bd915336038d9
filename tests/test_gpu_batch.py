"""Batched VQE energies (nwq_batch_*) against the oracle, per parameter set."""
import numpy as np
import pytest

import oracle
from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.sim import Batch, State

pytestmark = pytest.mark.gpu
H_LIST = (0.5, 1.0, 2.0)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2401_06861_gb300 import build
    build.build()
    yield


def tfim_energy_template(n, gates, pidx):
    """Terms Z_iZ_{i+1} and X_i with one energy row per h in H_LIST."""
    terms = inputs.zz_terms(n) + inputs.x_terms(n)
    coeffs = np.array([[-1.0] * (n - 1) + [-h] * n for h in H_LIST])
    return dict(n=n, gates=gates, param_index=pidx, terms=terms, coeffs=coeffs)


def oracle_energies(n, gates, pidx, params):
    g = [(name, q, (params[k],) if k >= 0 else prm) for (name, q, prm), k in zip(gates, pidx)]
    psi = oracle.sv_run(n, g)
    out = []
    for h in H_LIST:
        t = inputs.tfim_terms(n, 1.0, h)
        out.append(oracle.energy(oracle.sv_expect(psi, n, t), t) / np.vdot(psi, psi).real)
    return np.array(out)


def rel(e, eref, n, h):
    return np.abs(e - eref) / np.maximum(np.abs(eref), (n - 1) + n * np.asarray(h))


@pytest.mark.parametrize("dtype", [L.F64, L.F32])
@pytest.mark.parametrize("n", [1, 5, 12])
def test_batch_hea_matches_oracle(n, dtype):
    import torch
    layers, nsets = 4, 24
    gates, pidx = inputs.hea_ansatz(n, layers)
    nparams = layers * 2 * n
    params = inputs.hea_params(n, layers, nsets, seed=4096)
    b = Batch([tfim_energy_template(n, gates, pidx)], nparams, dtype)
    p = torch.from_numpy(params).cuda()
    out = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
    b.run(p.data_ptr(), nsets, out.data_ptr(), stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = np.array([oracle_energies(n, gates, pidx, params[s]) for s in range(nsets)])
    err = rel(got, ref, n, np.array(H_LIST)[None, :]).max()
    print(f"batch hea n={n} dtype={dtype}: max rel energy err {err:.3e}")
    assert err <= (1e-12 if dtype == L.F64 else 1e-6)
    b.close()


def test_batch_uneven_templates_in_one_launch_and_graph_replay():
    import torch
    specs = []
    for n, layers in ((4, 2), (9, 3), (13, 2)):
        g, pidx = inputs.hea_ansatz(n, layers)
        specs.append((n, g, pidx, layers * 2 * n))
    # a Trotter template with fixed angles (no parameters) as the fourth
    g4 = inputs.tfim_trotter(7, 1.0, 1.0, 0.05, 6)
    specs.append((7, g4, [-1] * len(g4), 0))
    nparams = max(s[3] for s in specs)
    b = Batch([tfim_energy_template(n, g, pidx) for n, g, pidx, _ in specs], nparams, L.F64)
    njobs = 40
    rng = np.random.default_rng(5)
    job_t = rng.integers(0, len(specs), njobs).astype(np.int32)
    stream = torch.cuda.current_stream().cuda_stream
    for it in range(2):  # second run: same pointers, new parameters -> graph replay
        params = rng.uniform(0, 2 * np.pi, (njobs, nparams))
        p = torch.from_numpy(params).cuda() if it == 0 else p.copy_(torch.from_numpy(params))
        jt = torch.from_numpy(job_t).cuda() if it == 0 else jt
        out = torch.zeros(njobs, 3, dtype=torch.float64, device="cuda") if it == 0 else out.zero_()
        b.run(p.data_ptr(), njobs, out.data_ptr(), job_template_ptr=jt.data_ptr(), stream=stream, graph=True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for j in range(njobs):
            n, g, pidx, _ = specs[job_t[j]]
            ref = oracle_energies(n, g, pidx, params[j])
            assert rel(got[j], ref, n, np.array(H_LIST)).max() <= 1e-12, (it, j)
    b.close()


def test_batch_equals_per_circuit_plain_path():
    import torch
    n, layers, nsets = 10, 3, 6
    gates, pidx = inputs.hea_ansatz(n, layers)
    params = inputs.hea_params(n, layers, nsets, seed=7)
    b = Batch([tfim_energy_template(n, gates, pidx)], layers * 2 * n, L.F64)
    p = torch.from_numpy(params).cuda()
    out = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
    b.run(p.data_ptr(), nsets, out.data_ptr(), stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for s in range(nsets):
        g = [(name, q, (params[s][k],) if k >= 0 else prm) for (name, q, prm), k in zip(gates, pidx)]
        with State(L.SV, n, L.F64) as st:
            st.apply(g, flags=L.PLAN_PLAIN)
            e = [st.expect(inputs.tfim_terms(n, 1.0, h), sum=True) for h in H_LIST]
        assert np.max(np.abs(got[s] - e)) <= 1e-12
    b.close()


def test_batch_energy_convenience_and_invalid_template_index():
    import torch
    n, layers, nsets = 6, 2, 5
    gates, pidx = inputs.hea_ansatz(n, layers)
    params = inputs.hea_params(n, layers, nsets, seed=9)
    t = tfim_energy_template(n, gates, pidx)
    garr, keep = L.encode_gates(gates, pidx)
    tarr = L.encode_terms(t["terms"])
    coeffs = np.ascontiguousarray(t["coeffs"]).reshape(-1)
    p = torch.from_numpy(params).cuda()
    out = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
    import ctypes
    L.check(L.lib().nwq_batch_energy(n, L.F64, garr, len(gates), ctypes.c_void_p(p.data_ptr()), nsets,
                                      layers * 2 * n, tarr, len(t["terms"]),
                                      coeffs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 3,
                                      ctypes.c_void_p(out.data_ptr()), None))
    ref = np.array([oracle_energies(n, gates, pidx, params[s]) for s in range(nsets)])
    assert rel(out.cpu().numpy(), ref, n, np.array(H_LIST)[None, :]).max() <= 1e-12
    # a job naming a template that does not exist gets NaN energies, the others are unaffected
    b = Batch([t], layers * 2 * n, L.F64)
    jt = torch.tensor([0, 3, 0, -1, 0], dtype=torch.int32, device="cuda")
    out2 = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
    b.run(p.data_ptr(), nsets, out2.data_ptr(), job_template_ptr=jt.data_ptr())
    torch.cuda.synchronize()
    o = out2.cpu().numpy()
    assert np.all(np.isnan(o[[1, 3]])) and np.allclose(o[[0, 2, 4]], ref[[0, 2, 4]], atol=1e-12)
    b.close()


def _mixed_template(n, seed):
    """Parametrised layers of one-qubit gates of every class (fixed, RX, RY,
    RZ, P, U3) between two-qubit gates (CX, CZ, SWAP, RZZ)."""
    rng = np.random.default_rng(seed)
    g, pidx, k = [], [], 0
    one = ["H", "S", "T", "SX", "RX", "RY", "RZ", "P", "U3"]
    two = ["CX", "CZ", "SWAP", "RZZ"]
    for _ in range(6):
        for q in range(n):
            for _ in range(int(rng.integers(1, 4))):
                name = one[int(rng.integers(len(one)))]
                prm = tuple(rng.uniform(-np.pi, np.pi, inputs.N_PARAMS.get(name, 0)))
                g.append(inputs.gate(name, (q,), prm))
                if name in ("RX", "RY", "RZ", "P"):
                    pidx.append(k)
                    k += 1
                else:
                    pidx.append(-1)
        for q in range(0, n - 1, 2 if rng.random() < 0.5 else 1):
            name = two[int(rng.integers(len(two)))]
            g.append(inputs.gate(name, (q, q + 1), (0.37,) if name == "RZZ" else ()))
            pidx.append(-1)
    return g, pidx, k


@pytest.mark.parametrize("dtype", [L.F64, L.F32])
def test_batch_shapes_agree_and_autotune(dtype):
    import torch
    tmpl, nps = [], []
    for i, n in enumerate((3, 7, 10)):
        g, pidx, k = _mixed_template(n, 50 + i)
        tmpl.append((n, g, pidx))
        nps.append(k)
    nparams, njobs = max(nps), 60
    params = np.random.default_rng(51).uniform(-np.pi, np.pi, (njobs, nparams))
    jt = np.arange(njobs, dtype=np.int32) % 3
    b = Batch([tfim_energy_template(n, g, pidx) for n, g, pidx in tmpl], nparams, dtype)
    s = torch.cuda.current_stream().cuda_stream
    p = torch.from_numpy(params).cuda()
    j = torch.from_numpy(jt).cuda()
    ref = np.array([oracle_energies(tmpl[t][0], tmpl[t][1], tmpl[t][2], params[i]) for i, t in enumerate(jt)])
    nref = np.array([tmpl[t][0] for t in jt])[:, None]
    tol = 1e-12 if dtype == L.F64 else 1e-6
    for fusion in (0, 1):
        for threads in (128, 256, 512):
            b.set_shape(threads, fusion)
            out = torch.zeros(njobs, 3, dtype=torch.float64, device="cuda")
            b.run(p.data_ptr(), njobs, out.data_ptr(), job_template_ptr=j.data_ptr(), stream=s, graph=True)
            torch.cuda.synchronize()
            err = rel(out.cpu().numpy(), ref, nref, np.array(H_LIST)[None, :]).max()
            assert err <= tol, (threads, fusion, err)
    out = torch.zeros(njobs, 3, dtype=torch.float64, device="cuda")
    best = b.autotune(p.data_ptr(), njobs, out.data_ptr(), job_template_ptr=j.data_ptr(), reps=2, stream=s)
    assert best["threads"] in (128, 256, 512) and best["fusion"] in (0, 1) and best["ms"] > 0
    out.zero_()
    b.run(p.data_ptr(), njobs, out.data_ptr(), job_template_ptr=j.data_ptr(), stream=s)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref, nref, np.array(H_LIST)[None, :]).max() <= tol
    print(f"batch autotune dtype={dtype}: {best}")
    for bad in ((64, 0), (256, 2)):
        with pytest.raises(L.NwqError):
            b.set_shape(*bad)
    b.close()


def test_batch_full_size_bench_configuration():
    # the benchmark's batched VQE at full size (n = 12, 4 layers, 4096 sets,
    # 3 energies, graph replay, autotuned kernel shape): a sample of sets
    # against the oracle and every energy above the exact ground energy
    import torch
    from scipy.sparse import csr_matrix
    from scipy.sparse.linalg import eigsh
    n, layers, nsets = 12, 4, 4096
    gates, pidx = inputs.hea_ansatz(n, layers)
    params = inputs.hea_params(n, layers, nsets, seed=4096)
    e0 = []
    N = 1 << n
    idx = np.arange(N)
    for h in H_LIST:  # H = -sum Z_i Z_{i+1} - h sum X_i as a sparse matrix
        diag = -sum(1.0 - 2.0 * (((idx >> i) ^ (idx >> (i + 1))) & 1) for i in range(n - 1))
        rows = np.concatenate([idx] + [idx for _ in range(n)])
        cols = np.concatenate([idx] + [idx ^ (1 << i) for i in range(n)])
        vals = np.concatenate([diag] + [np.full(N, -h) for _ in range(n)])
        e0.append(eigsh(csr_matrix((vals, (rows, cols)), shape=(N, N)), k=1, which="SA")[0][0])
    e0 = np.array(e0)
    s = torch.cuda.current_stream().cuda_stream
    p = torch.from_numpy(params).cuda()
    sample = np.random.default_rng(4097).choice(nsets, 24, replace=False)
    ref = np.array([oracle_energies(n, gates, pidx, params[i]) for i in sample])
    for dtype, tol in ((L.F64, 1e-12), (L.F32, 1e-6)):
        b = Batch([tfim_energy_template(n, gates, pidx)], layers * 2 * n, dtype, stream=s)
        out = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
        b.autotune(p.data_ptr(), nsets, out.data_ptr(), reps=1, stream=s)
        for _ in range(2):
            b.run(p.data_ptr(), nsets, out.data_ptr(), stream=s, graph=True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert rel(got[sample], ref, n, np.array(H_LIST)[None, :]).max() <= tol
        assert np.all(got >= e0[None, :] - 1e-6)
        b.close()


@pytest.mark.parametrize("fp64_pipe", [False, True])
def test_batch_fp64_double_words_and_fp64_pipe_match_the_oracle(fp64_pipe):
    # FP64 batches run in double words by default and on the FP64 pipe with
    # NWQ_BATCH_FP64_PIPE: every gate class (mixed templates), every kernel
    # shape, norms written, against the oracle at 1e-12
    import torch
    tmpl, nps = [], []
    for i, n in enumerate((2, 6, 9, 12)):
        g, pidx, k = _mixed_template(n, 70 + i)
        tmpl.append((n, g, pidx))
        nps.append(k)
    nparams, njobs = max(nps), 48
    params = np.random.default_rng(71).uniform(-np.pi, np.pi, (njobs, nparams))
    jt = np.arange(njobs, dtype=np.int32) % len(tmpl)
    b = Batch([tfim_energy_template(n, g, pidx) for n, g, pidx in tmpl], nparams, L.F64)
    s = torch.cuda.current_stream().cuda_stream
    p = torch.from_numpy(params).cuda()
    j = torch.from_numpy(jt).cuda()
    ref = np.array([oracle_energies(tmpl[t][0], tmpl[t][1], tmpl[t][2], params[i]) for i, t in enumerate(jt)])
    nref = np.array([tmpl[t][0] for t in jt])[:, None]
    for fusion in (0, 1):
        for threads in (128, 256, 512):
            b.set_shape(threads, fusion)
            out = torch.zeros(njobs, 3, dtype=torch.float64, device="cuda")
            norms = torch.zeros(njobs, dtype=torch.float64, device="cuda")
            b.run(p.data_ptr(), njobs, out.data_ptr(), job_template_ptr=j.data_ptr(), norms_ptr=norms.data_ptr(),
                  stream=s, fp64_pipe=fp64_pipe)
            torch.cuda.synchronize()
            err = rel(out.cpu().numpy(), ref, nref, np.array(H_LIST)[None, :]).max()
            assert err <= 1e-12, (threads, fusion, err)
            assert np.max(np.abs(norms.cpu().numpy() - 1.0)) <= 1e-12
    b.close()


@pytest.mark.parametrize("dtype,n", [(L.F64, 13), ("f64_pipe", 13), (L.F32, 14)])
def test_batch_at_the_largest_qubit_counts(dtype, n):
    # the largest states the batched kernel takes (shared memory: 2^13 x 16 bytes
    # FP64 or double words, 2^14 x 8 bytes FP32), every kernel shape, against the oracle
    import torch
    pipe = dtype == "f64_pipe"
    dtype = L.F64 if pipe else dtype
    layers, nsets = 2, 6
    gates, pidx = inputs.hea_ansatz(n, layers)
    params = inputs.hea_params(n, layers, nsets, seed=4100 + n)
    b = Batch([tfim_energy_template(n, gates, pidx)], layers * 2 * n, dtype)
    p = torch.from_numpy(params).cuda()
    ref = np.array([oracle_energies(n, gates, pidx, params[s]) for s in range(nsets)])
    for fusion in (0, 1):
        for threads in (128, 256, 512):
            b.set_shape(threads, fusion)
            out = torch.zeros(nsets, 3, dtype=torch.float64, device="cuda")
            b.run(p.data_ptr(), nsets, out.data_ptr(), fp64_pipe=pipe)
            torch.cuda.synchronize()
            err = rel(out.cpu().numpy(), ref, n, np.array(H_LIST)[None, :]).max()
            assert err <= (1e-12 if dtype == L.F64 else 1e-6), (threads, fusion, err)
    b.close()
    with pytest.raises(L.NwqError):  # one qubit more does not fit
        Batch([tfim_energy_template(n + 1, *inputs.hea_ansatz(n + 1, 1))], 2 * (n + 1), dtype)
