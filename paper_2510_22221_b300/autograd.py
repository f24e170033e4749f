"""torch.autograd.Function over the library's checkpointed run and adjoint
(arxiv 2510.22221, section "Numerical Model"): the probe objective
J = sum over steps n >= n0 of |E(probe)|^2 as a differentiable function of
eps_r in the design box and of |H_bias|.  Argument marshalling only: the
forward run and the reverse sweep are the library's."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .solver import FdtdLlg


def _solver(w, eps_design: np.ndarray, h0: float, nsteps: int, llg_fixed_iter: int):
    from . import configure

    u = np.asarray(w.hbias, dtype=np.float64)
    nrm = np.linalg.norm(u)
    u = u / nrm if nrm > 0 else np.array([0.0, 0.0, 1.0])
    wd = dataclasses.replace(w, eps_design=np.asarray(eps_design, dtype=np.float64), hbias=h0 * u)
    sim = FdtdLlg.create(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, courant_factor=w.courant, probe_capacity=nsteps,
                         llg_fixed_iter=llg_fixed_iter)
    configure(sim, wd)
    return sim


class ProbeEnergy(torch.autograd.Function):
    """J(eps_design, h0) for workload w (its design box, sources and probes),
    run for nsteps steps; gradients by the library's adjoint with
    checkpoints every `interval` steps (0: sqrt(nsteps))."""

    @staticmethod
    def forward(ctx, eps_design, h0, w, nsteps: int, n0: int, interval: int = 0, llg_fixed_iter: int = 3):
        eps = eps_design.detach().cpu().numpy().astype(np.float64)
        sim = _solver(w, eps, float(h0), nsteps, llg_fixed_iter)
        sim.run_checkpointed(nsteps, interval)
        rows = np.stack([sim.probe(p)[:, :3] for p in range(len(w.probes))], axis=1)
        ctx.sim, ctx.rows, ctx.n0, ctx.shape = sim, rows, n0, eps.shape
        return torch.tensor(float((rows[n0:] ** 2).sum()), dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        seed = np.zeros_like(ctx.rows)
        seed[ctx.n0:] = 2.0 * ctx.rows[ctx.n0:] * float(gJ)
        ge, gh = ctx.sim.adjoint_step(seed, design_shape=ctx.shape)
        ctx.sim.destroy()
        ctx.sim = None
        return torch.from_numpy(ge), torch.tensor(gh, dtype=torch.float64), None, None, None, None, None


def probe_energy(w, eps_design, h0, nsteps: int, n0: int, interval: int = 0, llg_fixed_iter: int = 3):
    return ProbeEnergy.apply(eps_design, h0, w, nsteps, n0, interval, llg_fixed_iter)
