"""Writes tests/golden/dm_noisy_tfim_n13.npz from the CPU oracle.

The workload is the noisy transverse-field Ising evolution of the paper's
density-matrix use case (Sec. III: TFIM chain under a device noise model of
depolarising, thermal-relaxation and readout noise), at the full 13-qubit
size of the density-matrix benchmark: J = h = 1, dt = 0.05, T1/T2 drawn from
seed 2401, one-qubit gates 35 ns with p1 = 1e-3, CX 300 ns with p2 = 1e-2,
2% readout error.  The Kraus-form oracle runs one Trotter step (49 gates,
each followed by its noise) from |0..0><0..0|, records the results, then a
second step from that state.

Stored per step (k = 1, 2):
  z{k}        <Z_i> for every qubit (13 values)
  tfim{k}     Tr(rho P) of the 25 TFIM terms (12 ZZ bonds, then 13 X_i)
  rho{k}      10^4 sampled entries rho[r, c] (complex128), at rows ``r`` and
              columns ``c`` (shared by both steps, drawn from seed 1313)
  probs{k}    the outcome distribution with 2% symmetric readout error

Only ``oracle`` and the seeded input generators are used.  Usage:
python tests/golden/make_dm_n13_golden.py [output.npz]; about 3 minutes per
step on 16 Neoverse V2 cores, 20 minutes on 8 x86 cores.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2401_06861_gb300 import inputs  # noqa: E402

N = 13
SAMPLES = 10000
OUT = os.path.join(HERE, "dm_noisy_tfim_n13.npz")


def main():
    gates, noise = inputs.dm_noisy_tfim(N, 1)
    rng = np.random.default_rng(1313)
    r = rng.integers(0, 1 << N, SAMPLES)
    c = rng.integers(0, 1 << N, SAMPLES)
    out = dict(n=N, r=r, c=c, seed_rows_cols=1313, noise_seed=2401, steps=2)
    rho = None
    for k in (1, 2):
        t0 = time.perf_counter()
        rho = oracle.dm_run(N, gates, noise, rho)
        out[f"z{k}"] = oracle.dm_expect(rho, N, inputs.z_terms(N))
        out[f"tfim{k}"] = oracle.dm_expect(rho, N, inputs.tfim_terms(N))
        out[f"rho{k}"] = rho[r, c]
        out[f"probs{k}"] = oracle.dm_probs(rho, N, noise["readout_e"])
        print(f"step {k}: {time.perf_counter() - t0:.1f} s, trace {np.trace(rho).real:.15f}", flush=True)
    np.savez(sys.argv[1] if len(sys.argv) > 1 else OUT, **out)


if __name__ == "__main__":
    main()
