"""torch.autograd wrapper of the fixed-count projection: forward is
hp_project (fixed_iters = k, guess phi_0), backward is hp_project_adjoint.
Both run in the library's kernels; this module only wires them to autograd."""
from __future__ import annotations

import torch

import paper_2109_09363_gb300 as hp


class ProjectFixed(torch.autograd.Function):
    """(u*, v*, phi_0) -> (u, v, p) with k masked Jacobi sweeps (Eq. 2-3)."""

    @staticmethod
    def forward(ctx, u_star, v_star, phi0, flags, hctx, k, dt, rho0):
        u = u_star.detach().clone().contiguous()
        v = v_star.detach().clone().contiguous()
        if int(k) > 0:
            prm = hp.ProjectParams(fixed_iters=int(k), dt=float(dt), rho0=float(rho0))
        else:  # zero sweeps: the cap is reached at k = 0
            prm = hp.ProjectParams(threshold=0.0, max_iters=0, dt=float(dt), rho0=float(rho0))
        out = hp.hp_project(hctx, u, v, flags, prm, phi0=phi0.detach().contiguous())
        ctx.save_for_backward(flags)
        ctx.hctx, ctx.k, ctx.dt, ctx.rho0 = hctx, int(k), float(dt), float(rho0)
        return u, v, out["p"]

    @staticmethod
    def backward(ctx, gu, gv, gp):
        (flags,) = ctx.saved_tensors
        B, ny, nx = flags.shape
        dev = flags.device
        if gu is None:
            gu = torch.zeros((B, ny, nx + 1), dtype=torch.float32, device=dev)
        if gv is None:
            gv = torch.zeros((B, ny + 1, nx), dtype=torch.float32, device=dev)
        gp = None if gp is None else gp.contiguous()
        gus, gvs, gphi = hp.hp_project_adjoint(ctx.hctx, gu.contiguous(), gv.contiguous(), gp,
                                               flags, ctx.k, ctx.dt, ctx.rho0)
        return gus, gvs, gphi, None, None, None, None, None


def project_fixed(u_star, v_star, phi0, flags, hctx, k, dt=1.0, rho0=1.0):
    return ProjectFixed.apply(u_star, v_star, phi0, flags, hctx, k, dt, rho0)
