"""VQE for the transverse-field Ising chain (paper Sec. III and Fig. 4: the
variational quantum eigensolver with the COBYLA minimiser, noise-free and with
the device noise model).

The optimiser minimises E(theta) = <H> over the hardware-efficient ansatz of
``inputs.hea_ansatz`` (per layer RY, RZ on every qubit, then a CX ladder), with
H = -J sum Z_i Z_{i+1} - h sum X_i on the open chain.  Energies come from the
CUDA library:

* ``NoiseFreeEnergy``: the batched kernel (one CTA per parameter set, FP64 or
  FP32 storage, FP64 accumulation, <H>/<psi|psi>); ``batch(thetas)`` evaluates
  many sets in one launch (the multi-start initial points).
* ``NoisyEnergy``: the density-matrix path: every ansatz gate followed by its
  depolarising and thermal-relaxation channels, then Tr(rho H).

``minimize`` accepts any callable energy, so the optimiser loop runs without a
GPU in tests.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from . import inputs


class NoiseFreeEnergy:
    """E(theta) of the n-qubit, ``layers``-layer ansatz through the batched kernel."""

    def __init__(self, n, layers, J=1.0, h=1.0, dtype=L.F64, max_sets=256):
        import torch

        from .sim import Batch
        self.torch = torch
        self.n, self.layers = n, layers
        self.gates, self.pidx = inputs.hea_ansatz(n, layers)
        self.nparams = 2 * n * layers
        self.terms = inputs.tfim_terms(n, J, h)
        coeffs = np.array([[t[2] for t in self.terms]])
        self.stream = torch.cuda.Stream()
        self.b = Batch([dict(n=n, gates=self.gates, param_index=self.pidx, terms=self.terms, coeffs=coeffs)],
                       self.nparams, dtype, stream=self.stream.cuda_stream)
        self.max_sets = max_sets
        self.dparams = torch.empty(max_sets, self.nparams, dtype=torch.float64, device="cuda")
        self.dout = torch.empty(max_sets, 1, dtype=torch.float64, device="cuda")
        self.hparams = torch.empty(max_sets, self.nparams, dtype=torch.float64).pin_memory()
        self.hout = torch.empty(max_sets, 1, dtype=torch.float64).pin_memory()
        self.nevals = 0

    def batch(self, thetas):
        torch = self.torch
        thetas = np.atleast_2d(np.asarray(thetas, np.float64))
        if thetas.shape[1] != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {thetas.shape[1]}")
        out = []
        for s in range(0, len(thetas), self.max_sets):
            chunk = thetas[s:s + self.max_sets]
            k = len(chunk)
            self.hparams[:k].copy_(torch.from_numpy(chunk))
            with torch.cuda.stream(self.stream):
                self.dparams[:k].copy_(self.hparams[:k], non_blocking=True)
                self.b.run(self.dparams.data_ptr(), k, self.dout.data_ptr(), stream=self.stream.cuda_stream)
                self.hout[:k].copy_(self.dout[:k], non_blocking=True)
            self.stream.synchronize()
            out.append(self.hout[:k, 0].numpy().copy())
        self.nevals += len(thetas)
        return np.concatenate(out)

    def __call__(self, theta):
        return float(self.batch(theta)[0])

    def close(self):
        self.b.close()


class NoisyEnergy:
    """E(theta) on the density matrix with the device noise model ``noise``
    (``inputs.noise_params``): each gate is followed by its noise channels."""

    def __init__(self, n, layers, noise, J=1.0, h=1.0, dtype=L.F64):
        from .sim import State
        self.n, self.layers, self.noise = n, layers, noise
        self.nparams = 2 * n * layers
        self.terms = inputs.tfim_terms(n, J, h)
        self.state = State(L.DM, n, dtype)
        self.nevals = 0

    def __call__(self, theta):
        theta = np.asarray(theta, np.float64)
        if theta.shape != (self.nparams,):
            raise ValueError(f"expected {self.nparams} parameters, got {theta.shape}")
        gates, _ = inputs.hea_ansatz(self.n, self.layers, theta)
        self.state.reset()
        self.state.apply(gates, noise=self.noise)
        self.nevals += 1
        return float(self.state.expect(self.terms, sum=True))

    def close(self):
        self.state.close()


def minimize(energy, nparams, x0=None, starts=1, batch_energy=None, seed=4096, maxiter=2000, rhobeg=0.5,
             tol=1e-6):
    """COBYLA on ``energy`` (theta -> float) from x0, or from the best of
    ``starts`` seeded random points in [0, 2 pi) (scored with ``batch_energy``
    in one call when given, else one by one).  Returns energy, theta, nfev,
    the energy of every evaluation (history) and scipy's success flag."""
    from scipy.optimize import minimize as sp_minimize
    if x0 is None:
        cand = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, size=(max(starts, 1), nparams))
        scores = batch_energy(cand) if batch_energy is not None else np.array([energy(c) for c in cand])
        x0 = cand[int(np.argmin(scores))]
    x0 = np.asarray(x0, np.float64)
    hist = []

    def f(theta):
        e = float(energy(theta))
        hist.append(e)
        return e

    res = sp_minimize(f, x0, method="COBYLA", options=dict(maxiter=maxiter, rhobeg=rhobeg, tol=tol))
    return dict(energy=float(res.fun), theta=np.asarray(res.x), nfev=int(res.nfev), history=np.array(hist),
                success=bool(res.success))
