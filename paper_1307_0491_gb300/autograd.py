"""torch.autograd.Function over many steps of the SVE scheme (the discrete
adjoint of libsve): gradients of any scalar function of the final bed with
respect to the initial bed z_b, the Grass constants A_g, m_g and the friction
coefficient (K for Strickler, f for Darcy-Weisbach), with the time steps of
the forward run recorded and held fixed.

    z_T = bed_evolution(z0, A_g, m_g, K, params, h0, hu0, hv0, nsteps)

z0, h0, hu0, hv0: CUDA float64 tensors (ny, nx); A_g, m_g, K: 0-dim float64
tensors.  Forward: sve_record_forward (checkpoints every ~sqrt(nsteps) steps);
backward: sve_adjoint.  Argument marshalling only; all arithmetic runs in
libsve's kernels.
"""
from __future__ import annotations

import torch

from . import sve


class _BedEvolution(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z0, A_g, m_g, K, params, h0, hu0, hv0, nsteps, checkpoint_every):
        p = dict(params)
        p["A_g"] = float(A_g)
        p["m_g"] = float(m_g)
        if p.get("friction") == "strickler":
            p["K_st"] = float(K)
        elif p.get("friction") == "darcy":
            p["f_dw"] = float(K)
        solver = sve.Solver(p, "fp64", stream=torch.cuda.current_stream().cuda_stream)
        solver.set_state(h0, hu0, hv0, z0)
        solver.record_forward(int(nsteps), int(checkpoint_every))
        zT = torch.empty_like(z0)
        hT, huT, hvT = torch.empty_like(z0), torch.empty_like(z0), torch.empty_like(z0)
        solver.get_state_device(hT, huT, hvT, zT)
        ctx.solver = solver
        return zT

    @staticmethod
    def backward(ctx, g_zT):
        solver = ctx.solver
        g = g_zT.contiguous()
        g_z0 = torch.empty_like(g)
        rc, gp = sve.sve_adjoint(solver.h, (None, None, None, g.data_ptr()), sve.SVE_DEVICE,
                                 (None, None, None, g_z0.data_ptr()))
        if rc:
            raise sve.SveError(rc, "sve_adjoint")
        dev = g.device
        t = lambda x: torch.tensor(x, dtype=torch.float64, device=dev)
        return g_z0, t(gp[0]), t(gp[1]), t(gp[2]), None, None, None, None, None, None


def bed_evolution(z0, A_g, m_g, K, params: dict, h0, hu0, hv0, nsteps: int, checkpoint_every: int = 0):
    """Bed elevation after nsteps CFL steps, differentiable in z0, A_g, m_g, K."""
    return _BedEvolution.apply(z0, A_g, m_g, K, params, h0, hu0, hv0, nsteps, checkpoint_every)
