"""torch.autograd wrapper of stokes_solve: the solution (u, p) as a
differentiable function of the nodal forcing f and the cell viscosities
nu_cell, with the backward pass through the library's discrete adjoint
(stokes_adjoint_solve, stokes_grad_viscosity).  Argument marshalling only:
setup, both solves and the gradient contraction run in the CUDA library.

Orders: f is [dim, n_vel_nodes] in the library's velocity-node order
(StokesMG.nodes()), nu_cell is [n_cells] in the finest-mesh order
(StokesMG.cell_centroids()); u is returned as [dim, n_vel_nodes] and p as
[n_pres_nodes].  The forward keeps its handle (and its device memory) until
the backward has run.

solve_batched is the same map for nrhs forcings at once (stokes_solve_batched
forward, stokes_adjoint_solve_batched and stokes_grad_viscosity_batched
backward): f is [nrhs, dim, n_vel_nodes], u [nrhs, dim, n_vel_nodes] and p
[nrhs, n_pres_nodes]; the viscosity gradient is summed over the columns.
"""
import numpy as np
import torch

from ._binding import BATCH_3XTF32, MIXED, StokesMG


class _StokesSolve(torch.autograd.Function):

    @staticmethod
    def forward(ctx, f, nu_cell, spec, tol):
        verts, cells, n_refine, family, k, kw = spec
        h = StokesMG(verts, cells, n_refine, family, k, nu_cell=np.ascontiguousarray(nu_cell.detach().cpu().numpy()),
                     **kw)
        u, p, _, _ = h.solve(f.detach().reshape(-1).contiguous(), tol=tol)
        ctx.h, ctx.tol, ctx.f_shape = h, tol, f.shape
        ctx.nu_device, ctx.nu_dtype = nu_cell.device, nu_cell.dtype
        ctx.save_for_backward(u)
        return u.view(f.shape), p

    @staticmethod
    def backward(ctx, gu, gp):
        h = ctx.h
        (u,) = ctx.saved_tensors
        gu = torch.zeros_like(u) if gu is None else gu.reshape(-1).to(torch.float64).contiguous()
        if gp is None:
            gp = torch.zeros(h.info()["n_pres_nodes"], dtype=torch.float64, device=u.device)
        gp = gp.to(torch.float64).contiguous()
        want_f, want_nu = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        lam_u, _, gf, _, _ = h.adjoint(gu, gp, tol=ctx.tol, grad_f=want_f)
        gnu = h.grad_viscosity(u, lam_u).to(device=ctx.nu_device, dtype=ctx.nu_dtype) if want_nu else None
        h.close()
        ctx.h = None
        return (gf.view(ctx.f_shape) if want_f else None), gnu, None, None


def solve(verts, cells, n_refine, family, k, f, nu_cell, tol=1e-10, **kw):
    """(u, p) = stokes_solve(f) on the handle set up with nu_cell, as a
    differentiable function of f (device float64 [dim, n_vel_nodes]) and
    nu_cell (float64 [n_cells]); extra keyword arguments go to StokesMG."""
    return _StokesSolve.apply(f, nu_cell, (verts, cells, n_refine, family, k, kw), tol)


class _StokesSolveBatched(torch.autograd.Function):

    @staticmethod
    def forward(ctx, F, nu_cell, spec, tol, mode):
        verts, cells, n_refine, family, k, kw = spec
        h = StokesMG(verts, cells, n_refine, family, k, nu_cell=np.ascontiguousarray(nu_cell.detach().cpu().numpy()),
                     **kw)
        nrhs = F.shape[0]
        U, Pp, _, _ = h.solve_batched(F.detach().reshape(nrhs, -1), mode=mode, tol=tol)
        ctx.h, ctx.tol, ctx.mode, ctx.f_shape = h, tol, mode, F.shape
        ctx.nu_device, ctx.nu_dtype = nu_cell.device, nu_cell.dtype
        ctx.save_for_backward(U)
        return U.view(F.shape), Pp

    @staticmethod
    def backward(ctx, gU, gP):
        h = ctx.h
        (U,) = ctx.saved_tensors
        nrhs = U.shape[0]
        gU = torch.zeros_like(U) if gU is None else gU.reshape(nrhs, -1).to(torch.float64).contiguous()
        if gP is None:
            gP = torch.zeros(nrhs, h.info()["n_pres_nodes"], dtype=torch.float64, device=U.device)
        gP = gP.to(torch.float64).contiguous()
        want_f, want_nu = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        LU, _, GF, _, _ = h.adjoint_batched(gU, gP, mode=ctx.mode, tol=ctx.tol, grad_f=want_f)
        gnu = h.grad_viscosity_batched(U, LU).to(device=ctx.nu_device, dtype=ctx.nu_dtype) if want_nu else None
        h.close()
        ctx.h = None
        return (GF.view(ctx.f_shape) if want_f else None), gnu, None, None, None


def solve_batched(verts, cells, n_refine, family, k, F, nu_cell, tol=1e-10, mode=BATCH_3XTF32, **kw):
    """(U, P) = stokes_solve_batched(F) on a MIXED handle set up with nu_cell,
    differentiable in F (device float64 [nrhs, dim, n_vel_nodes]) and nu_cell
    (float64 [n_cells]); extra keyword arguments go to StokesMG."""
    kw.setdefault("precision", MIXED)
    return _StokesSolveBatched.apply(F, nu_cell, (verts, cells, n_refine, family, k, kw), tol, mode)
