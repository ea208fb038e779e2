"""Discrete adjoint of the Stokes solve with respect to the forcing and the
cell-wise viscosity.  Oracle: test infrastructure (only tests/, the smoke
entry and bench's CPU legs use it).

Forward map (Sec. 2, Eq. 2.2-2.3, with nu_e constant on each cell e):
    K(nu) x = b(f, nu) on the free DoFs, K = [A(nu) B^T; B 0],
    A(nu) = sum_e nu_e A_e (A_e the cell's unit-viscosity vector Laplacian),
    b = F - K_full[free, D] g with F_c = M_v f_c (nodal forcing, exact mass
    product), u = g on the boundary, and the pressure normalised to
    int p = 0 afterwards: p_out = Pi p, Pi = I - 1 w^T / (w^T 1), w_j = int psi_j.
For a loss L(u, p_out), with gu = dL/du (all velocity nodes) and
gp = dL/dp_out, the adjoint lambda solves K^T lambda = r, where
    r = (gu on the free velocity DoFs, Pi^T gp).
K is symmetric, and r is orthogonal to its null space (the constant
pressures), so lambda exists.  Its pressure part is fixed only up to a
constant, which the gradients below never see.  Extend lambda by zero on
the Dirichlet DoFs; then
    dL/df_c  = M_v lambda_u,c                (b_u = M_v f on the free rows)
    dL/dnu_e = -lambda_u,e^T A_e u_e         (d b / d nu_e = -dK_full/dnu_e [.,D] g,
                                              so the lifting folds into the full u)
with u_e the element vector of the full velocity, boundary values included.
The paper does not differentiate its solver; this is the standard adjoint
of a linear solve, written for the discretisation of oracle.stokes.

Parity unpinned by the paper (it prints no gradients).  The pins are central
finite differences of the forward map and the symmetry of K
(tests/test_oracle_adjoint.py).
"""
import numpy as np

from . import stokes


def forward(disc: stokes.Discretization, f_nodal, g_nodal=None):
    """Full solution (u with boundary values, p with int p = 0) by the
    bordered sparse direct solve."""
    b, xD = stokes.load_vector(disc, f_nodal, g_nodal)
    x = stokes.direct_solve(disc, b)
    return stokes.zero_mean_pressure(disc, stokes.expand(disc, x, xD))


def adjoint_rhs(disc: stokes.Discretization, gu, gp):
    """r = dL/dx on the free DoFs: gu on the free velocity DoFs, Pi^T gp on
    the pressures."""
    d, nV = disc.d, disc.V.n
    g = np.zeros(disc.n_full)
    g[:d * nV] = np.asarray(gu, dtype=np.float64).reshape(-1)
    w = disc.p_integrals
    gp = np.asarray(gp, dtype=np.float64)
    g[d * nV:] = gp - w * (gp.sum() / w.sum())
    return g[disc.free]


def adjoint(disc: stokes.Discretization, gu, gp):
    """lambda on the full DoF vector (zero on the Dirichlet DoFs; pressure
    shifted to zero plain mean)."""
    r = adjoint_rhs(disc, gu, gp)
    lam_free = stokes.direct_solve(disc, r)       # K symmetric: K^T lambda = K lambda
    lam = np.zeros(disc.n_full)
    lam[disc.free] = lam_free
    d, nV = disc.d, disc.V.n
    lam[d * nV:] -= lam[d * nV:].mean()
    return lam


def grad_forcing(disc: stokes.Discretization, lam):
    """dL/df [d, nV] = M_v lambda_u,c per component."""
    d, nV = disc.d, disc.V.n
    return np.stack([disc.Mv @ lam[c * nV:(c + 1) * nV] for c in range(d)])


def grad_viscosity(disc: stokes.Discretization, x_full, lam):
    """dL/dnu_e = -sum_c lambda_c[e]^T S_e u_c[e] for every cell e, S_e the
    unit-viscosity scalar stiffness of the cell."""
    d, nV = disc.d, disc.V.n
    S, _, _, _ = stokes.element_matrices(disc.verts, disc.cells, disc.k, disc.k - 1, d)
    cn = disc.V.cell_nodes
    g = np.zeros(len(disc.cells))
    for c in range(d):
        ue = x_full[c * nV:(c + 1) * nV][cn]        # [nc, nb]
        le = lam[c * nV:(c + 1) * nV][cn]
        g -= np.einsum("ea,eab,eb->e", le, S, ue)
    return g


def gradients(disc: stokes.Discretization, x_full, gu, gp):
    """(lambda, dL/df, dL/dnu) for the loss gradient (gu, gp) at x_full."""
    lam = adjoint(disc, gu, gp)
    return lam, grad_forcing(disc, lam), grad_viscosity(disc, x_full, lam)
