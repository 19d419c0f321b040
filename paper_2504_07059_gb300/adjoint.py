"""Gradients of a mole-fraction misfit through the C ABI's discrete adjoint.

``MoleFractionMisfit.apply(d_pairs, g, problem)`` returns the loss
L = sum_i sum_y (xbar_i(y) - target_i(y))^2 after ``problem.nsteps`` steps,
xbar the mean over x of the mole fractions, as a differentiable function of
the Maxwell-Stefan diffusivities ``d_pairs`` (one per species pair i < j, in
the order (0,1), (0,2), ..., (1,2), ...) and the body force ``g`` (g_x, g_y).
The forward pass runs ``evd_loss_gradient`` (D2Q9; its forward steps in FP64 or
FP32, the reverse sweep in FP64), which returns the
exact gradient of the discrete step together with the loss; the backward
pass scales it.  Argument marshalling only: the steps and their adjoint run
in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import evd


@dataclass
class Problem:
    shape: tuple            # (nx, ny)
    wall_mask: int
    molar_mass: tuple
    tau1: float
    x0: np.ndarray          # [ns][1][ny][nx] initial mole fractions
    target: np.ndarray      # [ns][ny] target row averages
    nsteps: int
    n0: np.ndarray | None = None
    checkpoint_every: int = 0
    mode: int = 0           # evd.EVD_ADJOINT_REVERSE (default) or evd.EVD_ADJOINT_DUAL
    forward: str = "fp64"   # storage of the forward pass: "fp64" or "fp32" (reverse sweep in FP64)


def pairs_to_matrix(ns: int, d_pairs) -> np.ndarray:
    D = np.zeros((ns, ns))
    k = 0
    for i in range(ns):
        for j in range(i + 1, ns):
            D[i, j] = D[j, i] = float(d_pairs[k])
            k += 1
    return D


def loss_and_gradient(problem: Problem, d_pairs, g):
    """(loss, dL/d d_pairs, dL/dg[:2]) as numpy values."""
    ns = len(problem.molar_mass)
    D = pairs_to_matrix(ns, d_pairs)
    sim = evd.Simulation(evd.EVD_D2Q9, problem.shape, problem.wall_mask, problem.molar_mass, D, problem.tau1,
                         (float(g[0]), float(g[1])), "fp64")
    try:
        x0 = np.ascontiguousarray(problem.x0, dtype=np.float64)
        n0 = None if problem.n0 is None else np.ascontiguousarray(problem.n0, dtype=np.float64)
        tgt = np.ascontiguousarray(problem.target, dtype=np.float64)
        evd.evd_set_adjoint_mode(sim.ctx, problem.mode)
        evd.evd_set_adjoint_forward(sim.ctx, problem.forward)
        loss, dD, dg = evd.evd_loss_gradient(sim.ctx, x0, tgt, problem.nsteps, n0, problem.checkpoint_every)
    finally:
        sim.close()
    dpairs = np.array([dD[i, j] for i in range(ns) for j in range(i + 1, ns)])
    return loss, dpairs, dg[:2].copy()


class MoleFractionMisfit(torch.autograd.Function):
    """L(D pairs, g) with its adjoint gradient (see the module docstring)."""

    @staticmethod
    def forward(ctx, d_pairs: torch.Tensor, g: torch.Tensor, problem: Problem):
        loss, dd, dg = loss_and_gradient(problem, d_pairs.detach().cpu().numpy(), g.detach().cpu().numpy())
        ctx.save_for_backward(torch.from_numpy(dd).to(d_pairs), torch.from_numpy(dg).to(g))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        dd, dg = ctx.saved_tensors
        return grad_out * dd, grad_out * dg, None
