"""Monolithic hMG / phMG V-cycle with Vanka-star additive Schwarz relaxation,
used as a right preconditioner of FGMRES.  Oracle: test infrastructure.

Follows, step by step and without blocking or fusion:
  * Eq. 3.1  two-grid error propagator (I-wMK)^nu2 (I-P K_c^-1 R K)(I-wMK)^nu1,
             applied recursively (Fig. 2) on the h-levels;
  * Eq. 3.2  defect-correction propagator on the p-levels, the low-order
             correction G_1 being n_V hMG cycles (Fig. 3, Fig. 6b);
  * Sec. 3.1 finite-element interpolation P, R = P^T, coarse operators by
             rediscretisation;
  * Eq. 3.4  additive Schwarz M^-1 = sum_i I_i^T W_i K_i^-1 I_i with
             ASMVankaStarPC patches (Sec. 3.4, Fig. 5): per mesh vertex the
             pressure DoFs of its star and the velocity DoFs of the closure of
             its star (SV: all pressure DoFs of the cells around it);
  * Sec. 4   Chebyshev(nu) around one ASM sweep, damping from an estimate
             of the largest eigenvalue of M^-1 K; exact coarsest solve;
             FGMRES(30) stopped on the relative 2-norm residual.

Readings of points the paper leaves open:
  * W_i = diag(1/m_j), m_j = number of patches containing DoF j.
  * Chebyshev interval [0.1, 1.1] * lambda_hat, lambda_hat = largest real
    part of the Ritz values of 15 Arnoldi steps on M^-1 K from a SplitMix64
    start vector (10 steps left the estimate on the P4 level ~10% low, so
    the interval missed the top of the spectrum).
  * nu_p sweeps on the p-levels, nu_h on every hMG level (including the
    finest-mesh P_2 level); n_V repeats only the hMG sub-cycle.
  * Coarsest solve: LU of K bordered by the zero-mean pressure constraint.
  * Dirichlet DoFs are removed from the system, the transfers and patches.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import geometry, lagrange, rng, stokes

TH, SV = stokes.TH, stokes.SV


def pmg_schedule(k: int):
    """Gradual p-coarsening schedule of Fig. 7 for the velocity degree:
    k in [2,5] -> P2;  k in [6,7] -> P4 -> P2;  k in [8,10] -> P5 -> P2."""
    if k <= 5:
        return [k, 2] if k > 2 else [2]
    if k <= 7:
        return [k, 4, 2]
    return [k, 5, 2]


def scalar_interpolation(Vc: stokes.Space, Vf: stokes.Space, fine_to_coarse_cell):
    """Finite-element interpolation of a coarse scalar Lagrange space into a
    nested fine one (Sec. 3.1): row j holds the coarse basis functions
    evaluated at fine node j, located in the coarse cell that contains the
    fine cell owning it.  Values with |v| <= 1e-14 are exact zeros of the
    rational lattice evaluation and are dropped."""
    d = Vc.d
    rows, cols, vals = [], [], []
    done = np.zeros(Vf.n, dtype=bool)
    for fc in range(len(Vf.cells)):
        nodes = Vf.cell_nodes[fc]
        todo = nodes[~done[nodes]]
        if len(todo) == 0:
            continue
        done[todo] = True
        cc = fine_to_coarse_cell[fc]
        lam = lagrange.to_barycentric(Vc.verts, Vc.cells[cc], Vf.coords[todo])
        val = lagrange.basis(Vc.k, d, lam)         # [m, nb_c]
        for a, fn in enumerate(todo):
            for b, cn in enumerate(Vc.cell_nodes[cc]):
                if abs(val[a, b]) > 1e-14:
                    rows.append(fn); cols.append(cn); vals.append(val[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(Vf.n, Vc.n))


def monolithic_interpolation(fine: stokes.Discretization, coarse: stokes.Discretization, f2c):
    """P = blockdiag(P_V, ..., P_V, P_Q) restricted to free fine rows and free
    coarse columns (Dirichlet rows/columns removed)."""
    PV = scalar_interpolation(coarse.V, fine.V, f2c)
    PQ = scalar_interpolation(coarse.Q, fine.Q, f2c)
    P = sp.block_diag([PV] * fine.d + [PQ]).tocsr()
    return P[fine.free][:, coarse.free].tocsr()


def vanka_star_patches(disc: stokes.Discretization):
    """ASMVankaStarPC patches (Sec. 3.4, Fig. 5): one per mesh vertex v.
    Velocity: every component of every node on the closure of star(v), i.e.
    all velocity nodes of the cells containing v.  Pressure: TH - nodes whose
    owning entity contains v (the star); SV - all pressure nodes of the cells
    containing v.  Dirichlet DoFs removed.  Returns a list of sorted arrays
    of free-DoF indices."""
    d, nV = disc.d, disc.V.n
    full_to_free = -np.ones(disc.n_full, dtype=np.int64)
    full_to_free[disc.free] = np.arange(disc.n_free)
    nverts = len(disc.verts)
    v2c = [[] for _ in range(nverts)]
    for ci, c in enumerate(disc.cells.tolist()):
        for v in c:
            v2c[v].append(ci)
    patches = []
    for v in range(nverts):
        cs = v2c[v]
        if not cs:
            continue
        vn = np.unique(disc.V.cell_nodes[cs].ravel())
        qn = np.unique(disc.Q.cell_nodes[cs].ravel())
        if disc.family == TH:
            qn = np.array([q for q in qn if v in disc.Q.entity[q]], dtype=np.int64)
        full = np.concatenate([c * nV + vn for c in range(d)] + [d * nV + qn])
        fr = full_to_free[full]
        fr = np.sort(fr[fr >= 0])
        if len(fr):
            patches.append(fr)
    return patches


class ASM:
    """Additive Schwarz M^-1 = sum_i I_i^T W_i K_i^-1 I_i (Eq. 3.4) with
    exact patch solves by partial-pivot LU (Sec. 3.4)."""

    def __init__(self, K: sp.csr_matrix, patches):
        self.patches = patches
        self.n = K.shape[0]
        mult = np.zeros(self.n)
        for p in patches:
            mult[p] += 1.0
        self.weight = np.where(mult > 0, 1.0 / np.maximum(mult, 1.0), 0.0)
        Kc = K.tocsr()
        self.blocks = [Kc[p][:, p].toarray() for p in patches]
        self.lu = [sla.lu_factor(B) for B in self.blocks]

    def apply(self, r):
        z = np.zeros(self.n)
        for p, lu in zip(self.patches, self.lu):
            y = sla.lu_solve(lu, r[p])
            z[p] += self.weight[p] * y
        return z


def arnoldi_lmax(K, Minv, v0, steps=10):
    """Largest real part of the Ritz values of `steps` Arnoldi steps (modified
    Gram-Schmidt) on M^-1 K from v0 (Sec. 4: the Chebyshev damping uses an
    estimate of the largest eigenvalue of M^-1 K)."""
    n = len(v0)
    m = min(steps, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v0 / np.linalg.norm(v0)
    used = m
    for j in range(m):
        w = Minv(K @ V[j])
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * abs(H[j, j]) + 1e-300:
            used = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    ritz = np.linalg.eigvals(H[:used, :used])
    return float(np.max(ritz.real))


def chebyshev(K, Minv, b, x, nu, lmax, lo=0.1, hi=1.1):
    """nu steps of Chebyshev iteration for K x = b preconditioned by M^-1 on
    the interval [lo, hi] * lmax (three-term recurrence of the scaled and
    shifted Chebyshev polynomials).  For nu = 1 from x = 0 this is
    x = 2/((lo+hi) lmax) M^-1 b, damped additive Schwarz."""
    a, bb = lo * lmax, hi * lmax
    theta, delta = (bb + a) / 2.0, (bb - a) / 2.0
    sigma = theta / delta
    rho = 1.0 / sigma
    x = x.copy()
    r = b - K @ x
    dvec = Minv(r) / theta
    for i in range(nu):
        x = x + dvec
        if i == nu - 1:
            break
        r = r - K @ dvec
        rho_new = 1.0 / (2.0 * sigma - rho)
        dvec = rho_new * rho * dvec + (2.0 * rho_new / delta) * Minv(r)
        rho = rho_new
    return x


@dataclass
class Level:
    disc: stokes.Discretization
    kind: str                   # "p" or "h" (relaxed levels) or "coarse"
    mesh_index: int
    asm: ASM = None
    lmax: float = None
    P: sp.csr_matrix = None     # interpolation from the next coarser level
    R: sp.csr_matrix = None     # restriction R = P^T


@dataclass
class Options:
    nu_p: int = 1
    nu_h: int = 1
    n_V: int = 1
    eig_steps: int = 15
    eig_seed: int = 0
    cheb_lo: float = 0.1
    cheb_hi: float = 1.1


class Hierarchy:
    """phMG hierarchy (Sec. 3.2, Fig. 3): p-levels on the finest mesh with the
    velocity degrees of `schedule` (first = k of the fine discretisation, the
    last = degree of every hMG level), then the hMG levels on the nested
    meshes down to the coarsest, solved exactly.  For SV the finest level is
    SV P_k on the Alfeld mesh and every coarser level is TH (Sec. 3.2: the
    gradual coarsening of SV goes through TH P_khat)."""

    def __init__(self, verts, cells, n_refine, family, schedule, barycentric=False,
                 nu_cells=None, opts: Options = None, lmax=None, eig_start=None):
        self.opts = opts or Options()
        meshes, parents = geometry.hierarchy(verts, cells, n_refine, barycentric)
        self.meshes, self.parents = meshes, parents
        self.levels = []
        npl = len(schedule) - 1
        # a cellwise viscosity is given on the finest mesh; a coarse cell takes
        # the mean of its children's values (reading for per-cell nu)
        nus = [None if nu_cells is None else np.asarray(nu_cells, dtype=np.float64)]
        for mi in range(len(meshes) - 1):
            if nus[-1] is None:
                nus.append(None)
                continue
            par = parents[mi]
            s = np.bincount(par, weights=nus[-1], minlength=len(meshes[mi + 1][1]))
            cnt = np.bincount(par, minlength=len(meshes[mi + 1][1]))
            nus.append(s / cnt)
        for i, deg in enumerate(schedule[:-1]):
            fam = family if i == 0 else TH
            self.levels.append(Level(stokes.discretize(*meshes[0], fam, deg, nus[0]), "p", 0))
        q = schedule[-1]
        for mi in range(len(meshes)):
            fam = family if (npl == 0 and mi == 0) else TH
            kind = "h" if mi < len(meshes) - 1 else "coarse"
            self.levels.append(Level(stokes.discretize(*meshes[mi], fam, q, nus[mi]), kind, mi))
        for i in range(len(self.levels) - 1):
            fine, coarse = self.levels[i], self.levels[i + 1]
            if fine.mesh_index == coarse.mesh_index:
                f2c = np.arange(len(fine.disc.cells))
            else:
                f2c = parents[fine.mesh_index]
            fine.P = monolithic_interpolation(fine.disc, coarse.disc, f2c)
            fine.R = fine.P.T.tocsr()
        for i, L in enumerate(self.levels[:-1]):
            L.asm = ASM(L.disc.K, vanka_star_patches(L.disc))
            if lmax is not None and lmax[i] is not None:
                L.lmax = float(lmax[i])
            else:
                n = L.disc.n_free
                v0 = eig_start[i] if eig_start is not None else rng.uniform_pm1(self.opts.eig_seed, i, np.arange(n))
                L.lmax = arnoldi_lmax(L.disc.K, L.asm.apply, v0, self.opts.eig_steps)
        self._coarse_setup()

    def _coarse_setup(self):
        """LU of the coarsest K bordered by c = (0, int psi_j) so that the
        coarse correction has zero-mean pressure (Sec. 4 uses a direct solve;
        Sec. 2 fixes p in L^2_0)."""
        disc = self.levels[-1].disc
        n = disc.n_free
        c = np.zeros(n)
        pm = disc.pressure_mask_free()
        c[pm] = disc.p_integrals[disc.free[pm] - disc.d * disc.V.n]
        Kb = np.zeros((n + 1, n + 1))
        Kb[:n, :n] = disc.K.toarray()
        Kb[:n, n] = c
        Kb[n, :n] = c
        self.coarse_bordered = Kb
        self.coarse_lu = sla.lu_factor(Kb)

    def coarse_solve(self, r):
        n = len(r)
        return sla.lu_solve(self.coarse_lu, np.concatenate([r, [0.0]]))[:n]

    def smooth(self, i, b, x, nu):
        L = self.levels[i]
        o = self.opts
        return chebyshev(L.disc.K, L.asm.apply, b, x, nu, L.lmax, o.cheb_lo, o.cheb_hi)

    def hcycle(self, i, r):
        """hMG V-cycle (Eq. 3.1, Fig. 2) for K_i e = r from e = 0."""
        if self.levels[i].kind == "coarse":
            return self.coarse_solve(r)
        L = self.levels[i]
        nu = self.opts.nu_h
        e = self.smooth(i, r, np.zeros_like(r), nu)
        rc = L.R @ (r - L.disc.K @ e)
        e = e + L.P @ self.hcycle(i + 1, rc)
        return self.smooth(i, r, e, nu)

    def cycle(self, i, r):
        """phMG defect-correction cycle (Eq. 3.2) on p-level i; on the first
        hMG level it runs n_V hMG cycles, each on the current defect."""
        L = self.levels[i]
        if L.kind != "p":
            e = np.zeros_like(r)
            for _ in range(self.opts.n_V):
                e = e + self.hcycle(i, r - L.disc.K @ e)
            return e
        nu = self.opts.nu_p
        e = self.smooth(i, r, np.zeros_like(r), nu)
        rc = L.R @ (r - L.disc.K @ e)
        e = e + L.P @ self.cycle(i + 1, rc)
        return self.smooth(i, r, e, nu)

    def vcycle(self, r):
        """z = B_MG r: one application of the preconditioner."""
        return self.cycle(0, np.asarray(r, dtype=np.float64))


def fgmres(K, b, precond, tol=1e-8, restart=30, maxit=1000, x0=None):
    """Right-preconditioned flexible GMRES(restart) with modified Gram-Schmidt
    Arnoldi and Givens rotations, stopped when ||b - K x||_2 <= tol ||b - K x0||_2
    (Sec. 4: FGMRES with Krylov space of at most 30).  Returns (x, iterations,
    history of relative residual estimates)."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    r = b - K @ x
    beta0 = np.linalg.norm(r)
    hist = [1.0]
    if beta0 == 0.0:
        return x, 0, hist
    its = 0
    beta = beta0
    while its < maxit:
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        converged = False
        j_end = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = K @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) <= tol * beta0 or its >= maxit:
                converged = abs(g[j + 1]) <= tol * beta0
                break
        y = sla.solve_triangular(H[:j_end, :j_end], g[:j_end])
        x = x + Z[:j_end].T @ y
        if converged:
            break
        r = b - K @ x
        beta = np.linalg.norm(r)
        if beta <= tol * beta0:
            break
    return x, its, hist


def solve(h: Hierarchy, f_nodal, g_nodal=None, tol=1e-8, restart=30, maxit=1000):
    """stokes_solve: load vector, lifting, FGMRES-phMG, zero-mean pressure."""
    disc = h.levels[0].disc
    b, xD = stokes.load_vector(disc, f_nodal, g_nodal)
    x, its, hist = fgmres(disc.K, b, h.vcycle, tol, restart, maxit)
    full = stokes.zero_mean_pressure(disc, stokes.expand(disc, x, xD))
    return full, its, hist, b, x
