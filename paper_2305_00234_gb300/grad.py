"""torch.autograd wrapper: F(rho) with the hand-written adjoint run as its backward.

forward  = fdtd_set_density + fdtd_forward (the library keeps the FP64 forward DFT over the
           design box as the only checkpoint: design voxels x 3 x F complex values);
backward = fdtd_adjoint + fdtd_gradient, scaled by the incoming gradient.

No time history is stored (the paper stores E and Q for every step over the design domain,
Sec. 2); `checkpoint_bytes` reports both sizes.
"""
from __future__ import annotations

import torch

from .problem import Problem


class FdtdGrad(torch.autograd.Function):
    """F = FdtdGrad.apply(rho, problem): rho is a (dnz, dny, dnx) float32/float64 CUDA tensor."""

    @staticmethod
    def forward(ctx, rho, problem):
        if not isinstance(problem, Problem):
            raise TypeError("problem must be a paper_2305_00234_gb300.Problem")
        problem.set_density(rho.detach().contiguous())
        F, _ = problem.forward()
        ctx.problem = problem
        ctx.version = problem.version       # the handle's density and forward DFT this node depends on
        ctx.rho_meta = (rho.shape, rho.dtype, rho.device)
        return torch.tensor(F, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad_F):
        p = ctx.problem
        if p.version != ctx.version:
            # the handle keeps one density and one forward DFT: a later forward on the same Problem
            # replaced the state this node's adjoint run needs
            raise RuntimeError("FdtdGrad.backward: the Problem ran another forward (or set another density) "
                               "after this one; run backward before the next forward on the same Problem, "
                               "or use one Problem per graph node")
        shape, dtype, device = ctx.rho_meta
        p.adjoint()
        g = torch.empty(shape, dtype=dtype if dtype in (torch.float32, torch.float64) else torch.float32,
                        device=device)
        if device.type == "cuda":
            p.gradient(g)
        else:
            import numpy as np
            g = torch.from_numpy(p.gradient(np.zeros(shape, dtype=np.float64))).to(dtype)
        return g * grad_F.to(g.dtype), None


class FilterProject(torch.autograd.Function):
    """rho_b = FilterProject.apply(rho, R, beta, eta): cone filter (Eq. (FilterFunction)) and smoothed
    Heaviside projection (Eq. (Projection)) on the GPU; backward is Eq. (GradientsFiltered)."""

    @staticmethod
    def forward(ctx, rho, R, beta, eta):
        from . import _native as N
        rho = rho.detach().contiguous().float()
        rho_t, rho_b = torch.empty_like(rho), torch.empty_like(rho)
        N.fdtd_filter_project(rho, rho_t, rho_b, R, beta, eta, torch.cuda.current_stream().cuda_stream)
        ctx.save_for_backward(rho_t)
        ctx.params = (R, beta, eta)
        return rho_b

    @staticmethod
    def backward(ctx, g):
        from . import _native as N
        (rho_t,) = ctx.saved_tensors
        out = torch.empty_like(rho_t)
        N.fdtd_filter_project_grad(rho_t, g.contiguous().float(), out, *ctx.params,
                                   torch.cuda.current_stream().cuda_stream)
        return out, None, None, None


def objective(rho, problem):
    """Differentiable F(rho)."""
    return FdtdGrad.apply(rho, problem)


def checkpoint_bytes(problem):
    """(DFT checkpoint bytes kept between forward and backward, bytes a full E + Q time history
    over the design box would take at the handle's precision)."""
    d = problem.desc
    ts = 4 if d["precision"] == 32 else 8
    nd = problem.nd
    dft = nd * 3 * problem.nf * 16
    per_step = sum(1 + 2 * p for p in problem.poles_total) * ts     # E plus complex Q per component
    history = nd * d["n_steps"] * per_step
    return dft, history
