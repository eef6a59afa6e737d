"""torch.autograd binding: effective coefficients of every level as a differentiable function
of the per-level kappa tensors. The forward pass calls mch_solve_level and
mch_effective_coeffs for each level, the backward pass mch_backward; the tensors only carry
the data (every computation runs in the library's kernels)."""
from __future__ import annotations

import torch

from ._mch import Solver


class HomogenizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver: Solver, labels: tuple, *kappas):
        Es = []
        for lev, (k, l) in enumerate(zip(kappas, labels), start=1):
            k = k.detach().contiguous()
            solver.solve_level(lev, k, l.contiguous())
            E = torch.empty((k.shape[0], solver.R, solver.R), dtype=torch.float64,
                            device=k.device)
            solver.effective_coeffs(lev, E)
            Es.append(E)
        ctx.solver = solver
        ctx.meta = [(k.shape, k.device) for k in kappas]
        return tuple(Es)

    @staticmethod
    def backward(ctx, *dEs):
        solver = ctx.solver
        dEs = [torch.zeros((shape[0], solver.R, solver.R), dtype=torch.float64, device=dev)
               if g is None else g.contiguous()
               for g, (shape, dev) in zip(dEs, ctx.meta)]
        grads = [torch.empty(shape, dtype=torch.float64, device=dev) for shape, dev in ctx.meta]
        solver.backward(dEs, grads)
        return (None, None, *grads)


def homogenize(solver: Solver, kappas, labels):
    """Effective coefficients (one [n_points, R, R] tensor per level) of the hierarchy, with
    kappa gradients through mch_backward. kappas[l] [n_points_l, n_l^2] float64 and
    labels[l] uint8 tensors on the solver's device."""
    return HomogenizeFn.apply(solver, tuple(labels), *kappas)
