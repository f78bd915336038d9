"""Writes the stored expected values under tests/golden/ from the CPU oracle.

Only ``oracle`` and the seeded input generators are used here.  The TFIM
trajectory follows the paper's first use case (Sec. III, Fig. 3: time
evolution of <sigma_z> of an n = 4 Ising chain); the paper plots it without
printing values, so this fixture is the oracle's own trajectory, pinned in
the test to the exact Trotter product of matrix exponentials.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2401_06861_gb300 import inputs  # noqa: E402


def tfim_n4():
    n, J, h, dt, steps = 4, 1.0, 1.0, 0.05, 40
    psi = oracle.zero_state(n)
    step = inputs.tfim_trotter(n, J, h, dt, 1)
    rows = []
    for _ in range(steps):
        psi = oracle.sv_run(n, step, psi)
        rows.append([float(v) for v in oracle.sv_expect(psi, n, inputs.z_terms(n))])
    return dict(source="oracle; use case of paper Sec. III / Fig. 3 (n=4 TFIM chain, <Z_i> vs time)",
                n=n, J=J, h=h, dt=dt, z=rows)


if __name__ == "__main__":
    with open(os.path.join(HERE, "tfim_n4_z_trajectory.json"), "w") as f:
        json.dump(tfim_n4(), f, indent=1)
