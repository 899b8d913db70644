"""torch.autograd binding of the hand-written adjoint.

``lbm_run(phi0, D, a, solver=..., nsteps=...)`` returns phi after ``nsteps``
steps; its backward runs the reverse-time CUDA kernels (lbm_cde_backward:
checkpoint-segment recompute + adjoint steps) and returns gradients with
respect to phi0, the diffusion tensor D (every entry treated as independent)
and the velocity field a(x) of u(x, t) = a(x) s(t).
"""
from __future__ import annotations

import torch


class LbmRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, D, a, solver, nsteps, sched, every):
        solver.set_D(D.detach().to(torch.float64).cpu().numpy())
        if a is not None:
            solver.set_velocity(a.detach(), None if sched is None else sched.detach())
        phiN = solver.forward_ckpt(phi0.detach(), int(nsteps), int(every))
        ctx.solver = solver
        ctx.has_a = a is not None
        ctx.D_meta = (D.dtype, D.device)
        return phiN

    @staticmethod
    def backward(ctx, g):
        want_da = ctx.has_a and ctx.needs_input_grad[2]
        dphi0, dD, _ds, da = ctx.solver.backward(g.contiguous(), want_da=want_da)
        dtype, device = ctx.D_meta
        dD_t = torch.from_numpy(dD).to(device=device, dtype=dtype)
        return dphi0, dD_t, da, None, None, None, None


def lbm_run(phi0, D, a=None, *, solver, nsteps, sched=None, every=0):
    """Differentiable run of ``solver`` (a paper_1404_2363_gb300.Solver with FP32
    storage) from phi0 for nsteps steps."""
    return LbmRun.apply(phi0, D, a, solver, nsteps, sched, every)
