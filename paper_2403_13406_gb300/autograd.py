"""Differentiable composite steps: a torch.autograd.Function over the C ABI.

forward(u0) runs n composite steps from equilibrium at u0 and returns the moments;
backward(dJ/du_T) calls eslbm_gradient, the hand-written reverse-mode kernels
(reverse shifts and transposed relaxation Jacobians, including the implicit
derivative of the entropic relaxation parameter) with checkpoints every K steps.
"""
import torch

from . import eslbm


class _Evolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, sim, n, K):
        sim.init_equilibrium(u0.detach())
        sim.step(n)
        uT = sim.moments()
        ctx.sim, ctx.n, ctx.K = sim, n, K
        ctx.save_for_backward(u0.detach())
        return uT

    @staticmethod
    def backward(ctx, g):
        (u0,) = ctx.saved_tensors
        du0 = ctx.sim.gradient(u0, g, ctx.n, ctx.K)
        return du0, None, None, None


def evolve(u0, sim, n, K=50):
    """Moments after n steps of ``sim``'s scheme from equilibrium at u0 (CUDA float64 tensor of
    shape (M, [ny,] nx)), differentiable with respect to u0."""
    if not isinstance(sim, eslbm.Simulation):
        raise TypeError("sim must be an eslbm.Simulation")
    return _Evolve.apply(u0, sim, int(n), int(K))
