"""ctypes binding of libstokes_mg.so (include/stokes_mg.h): argument
marshalling only.  Every numerical step runs inside the CUDA library; if the
library is missing or fails to load this module raises instead of falling
back to anything else."""
import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_ulonglong, c_void_p

import numpy as np

TH, SV = 0, 1
HIER_DIRECT, HIER_GRADUAL, HIER_EXPLICIT, HIER_HMG = 0, 1, 2, 3
FP64, MIXED = 0, 1
ERRORS = {-1: "EINVAL", -2: "EOOM", -3: "ESINGULAR", -4: "ENOTCONVERGED", -5: "ENONFINITE",
          -6: "ECUDA", -7: "EUNSUPPORTED"}
PROF_PATCH, PROF_SPMV, PROF_GJ, PROF_PULL, PROF_TRANSFER = 0, 1, 2, 3, 4
MAX_LEVELS = 16
BATCH_TF32, BATCH_3XTF32 = 0, 1
BATCH_MAX = 64


class Mesh(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n_verts", c_int), ("n_cells", c_int),
                ("verts", POINTER(c_double)), ("cells", POINTER(c_int))]


class Opts(ctypes.Structure):
    _fields_ = [("hierarchy", c_int), ("n_schedule", c_int), ("schedule", c_int * 8),
                ("nu_p", c_int), ("nu_h", c_int), ("n_V", c_int), ("eig_steps", c_int),
                ("eig_seed", c_ulonglong), ("cheb_lo", c_double), ("cheb_hi", c_double),
                ("lmax_override", c_double * 16), ("precision", c_int), ("restart", c_int),
                ("maxit", c_int), ("use_graph", c_int), ("host_only", c_int), ("prof_mask", c_int),
                ("patch_solver", c_int), ("batch_tune", c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_levels", c_int), ("dim", c_int), ("family", c_int), ("k", c_int),
                ("n_free", c_int * MAX_LEVELS), ("degree", c_int * MAX_LEVELS),
                ("level_family", c_int * MAX_LEVELS), ("mesh_index", c_int * MAX_LEVELS),
                ("is_p_level", c_int * MAX_LEVELS), ("nnz", c_longlong * MAX_LEVELS),
                ("n_patches", c_int * MAX_LEVELS), ("max_patch", c_int * MAX_LEVELS),
                ("patch_entries", c_longlong * MAX_LEVELS), ("lmax", c_double * MAX_LEVELS),
                ("n_vel_nodes", c_int), ("n_pres_nodes", c_int), ("singular_patch", c_int),
                ("t_mesh_ms", c_double), ("t_assembly_ms", c_double), ("t_upload_ms", c_double),
                ("t_gather_lu_ms", c_double), ("t_coarse_ms", c_double), ("t_eig_ms", c_double),
                ("t_graph_ms", c_double), ("t_total_ms", c_double), ("kernel_launches", c_longlong),
                ("t_spaces_ms", c_double), ("t_matrices_ms", c_double), ("t_patches_ms", c_double),
                ("t_transfers_ms", c_double), ("t_launch_thread_ms", c_double),
                ("t_launch_wait_ms", c_double), ("t_upload_post_ms", c_double)]


class StokesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libstokes_mg.so")


def lib():
    """Load the CUDA library (building it first if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        from . import build
        build.build()
    L = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "stokes_mg_default_opts": (None, [POINTER(Opts)]),
        "stokes_mg_setup": (c_int, [POINTER(Mesh), c_int, c_int, c_int, c_int, POINTER(Opts), P, P, POINTER(P)]),
        "stokes_fbf_setup": (c_int, [POINTER(Mesh), c_int, c_int, POINTER(Opts), P, P, POINTER(P)]),
        "stokes_fbf_apply": (c_int, [P, P, P, P]),
        "stokes_mg_vcycle": (c_int, [P, P, P, c_int, P]),
        "stokes_mg_vcycle_batched": (c_int, [P, P, P, c_int, c_int, P]),
        "stokes_batch_plan": (c_int, [P, c_int, c_int, c_int, POINTER(c_int), P, P, P, P, P, P, POINTER(c_double)]),
        "stokes_adjoint_solve": (c_int, [P, P, P, c_double, c_double, P, P, P, P, P, P]),
        "stokes_fgmres_batched": (c_int, [P, P, P, c_int, c_int, c_double, P, P, P]),
        "stokes_selftest_bounded_wait": (c_int, [c_longlong, P]),
        "stokes_probe_fp64_peak": (c_int, [c_longlong, c_int, POINTER(c_double), POINTER(ctypes.c_float), P]),
        "stokes_grad_viscosity": (c_int, [P, P, P, P, P]),
        "stokes_solve_batched": (c_int, [P, P, P, c_int, c_int, c_double, c_double, P, P, P, P, P]),
        "stokes_adjoint_solve_batched": (c_int, [P, P, P, c_int, c_int, c_double, c_double, P, P, P, P, P, P]),
        "stokes_grad_viscosity_batched": (c_int, [P, P, P, c_int, P, P]),
        "stokes_mg_cell_centroids": (c_int, [P, P, P]),
        "stokes_solve": (c_int, [P, P, P, c_double, c_double, P, P, POINTER(c_int), POINTER(c_double), P]),
        "stokes_mg_info": (c_int, [P, POINTER(Stats)]),
        "stokes_mg_level_dofs": (c_int, [P, c_int, P, P, P]),
        "stokes_mg_nodes": (c_int, [P, P, P, P]),
        "stokes_mg_get_csr": (c_int, [P, c_int, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_longlong), P, P, P]),
        "stokes_mg_get_patches": (c_int, [P, c_int, POINTER(c_int), POINTER(c_longlong), P, P]),
        "stokes_mg_patch_matrices": (c_int, [P, c_int, P, P]),
        "stokes_mg_patch_inverses": (c_int, [P, c_int, P, P]),
        "stokes_mg_arnoldi_lmax": (c_int, [P, c_int, P, c_int, POINTER(c_double), P]),
        "stokes_mg_residual": (c_int, [P, c_int, P, P, P, c_int, P]),
        "stokes_mg_asm": (c_int, [P, c_int, P, P, c_int, P]),
        "stokes_mg_transfer": (c_int, [P, c_int, c_int, P, P, c_int, P]),
        "stokes_mg_coarse_solve": (c_int, [P, P, P, P]),
        "stokes_mg_fgmres": (c_int, [P, P, P, c_double, POINTER(c_int), POINTER(c_double), P]),
        "stokes_prof_enable": (c_int, [P, c_int, c_int]),
        "stokes_prof_read": (c_int, [P, c_int, POINTER(c_longlong), POINTER(c_double)]),
        "stokes_prof_read_one": (c_int, [P, c_int, c_longlong, POINTER(c_double)]),
        "stokes_mg_destroy": (None, [P]),
        "stokes_last_error": (ctypes.c_char_p, []),
        "stokes_batched_inverse_noalloc": (c_int, [c_int, P, P, POINTER(c_int), P]),
        "stokes_noalloc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def check(rc):
    if rc != 0:
        raise StokesError(rc, lib().stokes_last_error().decode())
    return rc


def default_opts(**kw):
    o = Opts()
    lib().stokes_mg_default_opts(byref(o))
    for k, v in kw.items():
        if k == "schedule":
            o.n_schedule = len(v)
            for i, x in enumerate(v):
                o.schedule[i] = int(x)
        elif k == "lmax_override":
            for i, x in enumerate(v):
                o.lmax_override[i] = float(x or 0.0)
        else:
            setattr(o, k, v)
    return o


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return c_void_p(t.data_ptr())


def _vin(t, n, what):
    """An input vector for the library: a contiguous float64 CUDA tensor with
    at least n elements (n None: no length check).  A tensor of another
    dtype, on the host or with gaps is converted first (on torch's current
    stream); one with too few elements raises ValueError, since the library
    would read past its end."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch.Tensor, got {type(t).__name__}")
    if n is not None and t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the library reads {n}")
    if not t.is_cuda:
        t = t.to(torch.device("cuda", torch.cuda.current_device()))
    if t.dtype != torch.float64:
        t = t.to(torch.float64)
    return t.contiguous()


def _vout(t, n, what):
    """An output (or in-out) vector: the library writes it in place, so it
    must already be a contiguous float64 CUDA tensor with at least n
    elements; anything else raises ValueError."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch.Tensor, got {type(t).__name__}")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{what}: must be a contiguous float64 CUDA tensor "
                         f"(got {t.dtype} on {t.device}, contiguous={t.is_contiguous()})")
    if n is not None and t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the library writes {n}")
    return t


def _rows(t):
    return 1 if t.dim() <= 1 else t.shape[0]


def _stream(stream):
    if stream is not None:
        return c_void_p(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def selftest_bounded_wait(polls=1000):
    """stokes_selftest_bounded_wait: 2 when the bounded mbarrier wait gives up
    and its kernel returns."""
    r = c_int()
    check(lib().stokes_selftest_bounded_wait(int(polls), byref(r)))
    return r.value


def probe_fp64_peak(iters=1 << 16, blocks_per_sm=2, stream=None):
    """stokes_probe_fp64_peak: (TFLOP/s, ms) of a timed DFMA-loop launch."""
    t, ms = c_double(), ctypes.c_float()
    check(lib().stokes_probe_fp64_peak(int(iters), int(blocks_per_sm), byref(t), byref(ms), _stream(stream)))
    return t.value, ms.value


class StokesMG:
    """Handle on a phMG hierarchy built by stokes_mg_setup."""

    def __init__(self, verts, cells, n_refine, family, k, barycentric=False, nu_cell=None,
                 stream=None, fbf=False, **opts):
        """fbf=True builds the FBF(phMG) solver of Eq. fbf instead
        (stokes_fbf_setup; Scott-Vogelius on the Alfeld-refined finest mesh)."""
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        self._mesh = Mesh(verts.shape[1], verts.shape[0], cells.shape[0],
                          verts.ctypes.data_as(POINTER(c_double)), cells.ctypes.data_as(POINTER(c_int)))
        self._keep = (verts, cells)
        self.opts = default_opts(**opts)
        nu = None
        if nu_cell is not None:
            nu = np.ascontiguousarray(nu_cell, dtype=np.float64)
            self._keep = self._keep + (nu,)
        self.h = c_void_p()
        self.stream = stream
        nu_p = None if nu is None else nu.ctypes.data_as(c_void_p)
        if fbf:
            if family != SV:
                raise ValueError("FBF is the Scott-Vogelius solver (family SV)")
            check(lib().stokes_fbf_setup(byref(self._mesh), int(n_refine), int(k), byref(self.opts), nu_p,
                                         _stream(stream), byref(self.h)))
        else:
            check(lib().stokes_mg_setup(byref(self._mesh), int(n_refine), int(bool(barycentric)), int(family), int(k),
                                        byref(self.opts), nu_p, _stream(stream), byref(self.h)))
        self.is_fbf = bool(fbf)
        self.dim = verts.shape[1]
        i = self.info()
        # vector lengths the ABI reads and writes (fixed once the handle exists)
        self._nfree = list(i["n_free"])
        self._nV = i["n_vel_nodes"]
        self._nQ = i["n_pres_nodes"]

    # ---- queries
    def info(self):
        s = Stats()
        check(lib().stokes_mg_info(self.h, byref(s)))
        nl = s.n_levels
        out = {}
        for name, _ in Stats._fields_:
            v = getattr(s, name)
            out[name] = list(v)[:nl] if isinstance(v, ctypes.Array) else v
        return out

    def level_dofs(self, level):
        n = self.info()["n_free"][level]
        xyz = np.zeros((n, self.dim))
        comp = np.zeros(n, dtype=np.int32)
        cc = np.zeros((n, self.dim))
        check(lib().stokes_mg_level_dofs(self.h, level, xyz.ctypes.data_as(c_void_p), comp.ctypes.data_as(c_void_p),
                                         cc.ctypes.data_as(c_void_p)))
        return xyz, comp, cc

    def nodes(self):
        i = self.info()
        vx = np.zeros((i["n_vel_nodes"], self.dim))
        px = np.zeros((i["n_pres_nodes"], self.dim))
        pc = np.zeros((i["n_pres_nodes"], self.dim))
        check(lib().stokes_mg_nodes(self.h, vx.ctypes.data_as(c_void_p), px.ctypes.data_as(c_void_p),
                                    pc.ctypes.data_as(c_void_p)))
        return vx, px, pc

    def get_csr(self, level, which=0):
        nr, nc, nnz = c_int(), c_int(), c_longlong()
        check(lib().stokes_mg_get_csr(self.h, level, which, byref(nr), byref(nc), byref(nnz), None, None, None))
        rp = np.zeros(nr.value + 1, dtype=np.int32)
        ci = np.zeros(nnz.value, dtype=np.int32)
        v = np.zeros(nnz.value)
        check(lib().stokes_mg_get_csr(self.h, level, which, byref(nr), byref(nc), byref(nnz),
                                      rp.ctypes.data_as(c_void_p), ci.ctypes.data_as(c_void_p), v.ctypes.data_as(c_void_p)))
        import scipy.sparse as sp
        return sp.csr_matrix((v, ci, rp), shape=(nr.value, nc.value))

    def patches(self, level):
        npch, nent = c_int(), c_longlong()
        check(lib().stokes_mg_get_patches(self.h, level, byref(npch), byref(nent), None, None))
        off = np.zeros(npch.value + 1, dtype=np.int32)
        dofs = np.zeros(nent.value, dtype=np.int32)
        check(lib().stokes_mg_get_patches(self.h, level, byref(npch), byref(nent), off.ctypes.data_as(c_void_p),
                                          dofs.ctypes.data_as(c_void_p)))
        return off, dofs

    # ---- device work (torch CUDA tensors, float64; inputs of another dtype
    # or on the host are converted, outputs are checked, see _vin / _vout)
    def vcycle(self, r, out=None):
        import torch
        nrhs = _rows(r)
        n = nrhs * self._nfree[0]
        r = _vin(r, n, "r")
        z = torch.empty_like(r) if out is None else _vout(out, n, "out")
        check(lib().stokes_mg_vcycle(self.h, _ptr(r), _ptr(z), nrhs, _stream(self.stream)))
        return z

    def fgmres_batched(self, B, mode=BATCH_TF32, tol=1e-8, out=None, raise_on_nonconv=True):
        """X with K X[c] = B[c] for the rows of B [nrhs, n_free] (device
        float64), by FGMRES-phMG in lockstep with the batched V-cycle
        (stokes_fgmres_batched).  Returns (X, iterations, relres [nrhs])."""
        import torch
        nrhs = _rows(B)
        B = _vin(B, nrhs * self._nfree[0], "B")
        X = torch.empty_like(B) if out is None else _vout(out, nrhs * self._nfree[0], "out")
        its = c_int()
        rel = np.zeros(nrhs, dtype=np.float64)
        rc = lib().stokes_fgmres_batched(self.h, _ptr(B), _ptr(X), nrhs, int(mode), float(tol), byref(its),
                                         rel.ctypes.data_as(c_void_p), _stream(self.stream))
        if rc != -4 or raise_on_nonconv:
            check(rc)
        return X, its.value, rel

    def batch_plan(self, level, mode=BATCH_TF32):
        """The batched patch GEMM's launches on a relaxed level
        (stokes_batch_plan): a list of dicts (kind, warps, count, lo, hi,
        us), and the one-launch-per-kind time in microseconds."""
        n = c_int()
        mx = 64
        arr = {k: np.zeros(mx, dtype=np.int32) for k in ("kind", "warps", "count", "lo", "hi")}
        us = np.zeros(mx, dtype=np.float64)
        single = c_double()
        check(lib().stokes_batch_plan(self.h, int(mode), int(level), mx, byref(n),
                                      *[arr[k].ctypes.data_as(c_void_p) for k in ("kind", "warps", "count", "lo", "hi")],
                                      us.ctypes.data_as(c_void_p), byref(single)))
        parts = [dict({k: int(arr[k][i]) for k in arr}, us=float(us[i])) for i in range(min(n.value, mx))]
        return parts, single.value

    def fbf_apply(self, r, out=None):
        """z = P^-1 r of Eq. fbf on the Stokes free DoFs (stokes_fbf_apply)."""
        import torch
        r = _vin(r, None, "r")
        z = torch.empty_like(r) if out is None else _vout(out, r.numel(), "out")
        check(lib().stokes_fbf_apply(self.h, _ptr(r), _ptr(z), _stream(self.stream)))
        return z

    def vcycle_batched(self, R, mode=BATCH_3XTF32, out=None):
        """Z = B_MG R for R of shape [nrhs, n_free] (float64, device), all
        right-hand sides in one interleaved pass (stokes_mg_vcycle_batched)."""
        import torch
        nrhs = _rows(R)
        R = _vin(R, nrhs * self._nfree[0], "R")
        Z = torch.empty_like(R) if out is None else _vout(out, nrhs * self._nfree[0], "out")
        check(lib().stokes_mg_vcycle_batched(self.h, _ptr(R), _ptr(Z), nrhs, int(mode), _stream(self.stream)))
        return Z

    def adjoint(self, gu, gp, nu=1.0, tol=1e-8, grad_f=True, raise_on_nonconv=True):
        """Discrete adjoint of solve (stokes_adjoint_solve): returns (lam_u,
        lam_p, dL/df or None, iterations, relres) for gu = dL/du [dim, nV]
        and gp = dL/dp [nQ] (device float64)."""
        import torch
        gu = _vin(gu, self.dim * self._nV, "gu")
        gp = _vin(gp, self._nQ, "gp")
        lam_u = torch.empty_like(gu)
        lam_p = torch.empty_like(gp)
        gf = torch.empty_like(gu) if grad_f else None
        its, rel = c_int(), c_double()
        rc = lib().stokes_adjoint_solve(self.h, _ptr(gu), _ptr(gp), float(nu), float(tol), _ptr(lam_u), _ptr(lam_p),
                                        _ptr(gf), byref(its), byref(rel), _stream(self.stream))
        if rc != -4 or raise_on_nonconv:
            check(rc)
        return lam_u, lam_p, gf, its.value, rel.value

    def grad_viscosity(self, u, lam_u):
        """dL/dnu per finest cell (stokes_grad_viscosity)."""
        import torch
        n = self.n_cells()
        u = _vin(u, self.dim * self._nV, "u")
        lam_u = _vin(lam_u, self.dim * self._nV, "lam_u")
        g = torch.empty(n, dtype=torch.float64, device=u.device)
        check(lib().stokes_grad_viscosity(self.h, _ptr(u), _ptr(lam_u), _ptr(g), _stream(self.stream)))
        return g

    def solve_batched(self, F, G=None, mode=BATCH_3XTF32, nu=1.0, tol=1e-8, raise_on_nonconv=True):
        """solve for nrhs forcings at once (stokes_solve_batched): F is
        [nrhs, dim * n_vel_nodes] device float64 (G the same shape or None).
        Returns (U [nrhs, dim * nV], P [nrhs, nQ], iterations, relres [nrhs])."""
        import torch
        nrhs = F.shape[0]
        F = _vin(F, nrhs * self.dim * self._nV, "F")
        G = None if G is None else _vin(G, nrhs * self.dim * self._nV, "G")
        nQ = self._nQ
        U = torch.empty_like(F)
        Pp = torch.empty(nrhs, nQ, dtype=torch.float64, device=F.device)
        its = c_int()
        rel = np.zeros(nrhs, dtype=np.float64)
        rc = lib().stokes_solve_batched(self.h, _ptr(F), _ptr(G), nrhs, int(mode), float(nu), float(tol), _ptr(U),
                                        _ptr(Pp), byref(its), rel.ctypes.data_as(c_void_p), _stream(self.stream))
        if rc != -4 or raise_on_nonconv:
            check(rc)
        return U, Pp, its.value, rel

    def adjoint_batched(self, GU, GP, mode=BATCH_3XTF32, nu=1.0, tol=1e-8, grad_f=True, raise_on_nonconv=True):
        """adjoint for nrhs loss gradients at once (stokes_adjoint_solve_batched):
        GU [nrhs, dim * nV], GP [nrhs, nQ].  Returns (LAM_U, LAM_P, dL/dF or
        None, iterations, relres [nrhs])."""
        import torch
        nrhs = GU.shape[0]
        GU = _vin(GU, nrhs * self.dim * self._nV, "GU")
        GP = _vin(GP, nrhs * self._nQ, "GP")
        LU = torch.empty_like(GU)
        LP = torch.empty_like(GP)
        GF = torch.empty_like(GU) if grad_f else None
        its = c_int()
        rel = np.zeros(nrhs, dtype=np.float64)
        rc = lib().stokes_adjoint_solve_batched(self.h, _ptr(GU), _ptr(GP), nrhs, int(mode), float(nu), float(tol),
                                                _ptr(LU), _ptr(LP), _ptr(GF), byref(its),
                                                rel.ctypes.data_as(c_void_p), _stream(self.stream))
        if rc != -4 or raise_on_nonconv:
            check(rc)
        return LU, LP, GF, its.value, rel

    def grad_viscosity_batched(self, U, LU):
        """sum over the rows of dL/dnu per finest cell
        (stokes_grad_viscosity_batched); U, LU [nrhs, dim * nV]."""
        import torch
        nrhs = U.shape[0]
        U = _vin(U, nrhs * self.dim * self._nV, "U")
        LU = _vin(LU, nrhs * self.dim * self._nV, "LU")
        g = torch.empty(self.n_cells(), dtype=torch.float64, device=U.device)
        check(lib().stokes_grad_viscosity_batched(self.h, _ptr(U), _ptr(LU), U.shape[0], _ptr(g),
                                                  _stream(self.stream)))
        return g

    def n_cells(self):
        nc = c_int()
        check(lib().stokes_mg_cell_centroids(self.h, byref(nc), None))
        return nc.value

    def cell_centroids(self):
        """[n_cells, dim] centroids of the finest cells, in nu_cell order."""
        nc = self.n_cells()
        x = np.zeros((nc, self.dim), dtype=np.float64)
        check(lib().stokes_mg_cell_centroids(self.h, byref(c_int()), x.ctypes.data_as(c_void_p)))
        return x

    def solve(self, f, g=None, nu=1.0, tol=1e-8, u=None, p=None, raise_on_nonconv=True):
        import torch
        nu_ = self.dim * self._nV
        f = _vin(f, nu_, "f")
        g = None if g is None else _vin(g, nu_, "g")
        u = torch.empty(nu_, dtype=torch.float64, device=f.device) if u is None else _vout(u, nu_, "u")
        p = torch.empty(self._nQ, dtype=torch.float64, device=f.device) if p is None else _vout(p, self._nQ, "p")
        its, rel = c_int(), c_double()
        rc = lib().stokes_solve(self.h, _ptr(f), _ptr(g), float(nu), float(tol), _ptr(u), _ptr(p),
                                byref(its), byref(rel), _stream(self.stream))
        if rc != 0 and (raise_on_nonconv or rc != -4):
            check(rc)
        return u, p, its.value, rel.value

    def fgmres(self, b, tol=1e-8):
        import torch
        b = _vin(b, self._nfree[0], "b")
        x = torch.empty_like(b)
        its, rel = c_int(), c_double()
        check(lib().stokes_mg_fgmres(self.h, _ptr(b), _ptr(x), float(tol), byref(its), byref(rel), _stream(self.stream)))
        return x, its.value, rel.value

    def patch_matrices(self, level):
        n = self.info()["patch_entries"][level]
        out = np.zeros(n)
        check(lib().stokes_mg_patch_matrices(self.h, level, out.ctypes.data_as(c_void_p), _stream(self.stream)))
        return out

    def patch_inverses(self, level):
        n = self.info()["patch_entries"][level]
        out = np.zeros(n)
        check(lib().stokes_mg_patch_inverses(self.h, level, out.ctypes.data_as(c_void_p), _stream(self.stream)))
        return out

    def arnoldi_lmax(self, level, v0, steps=10):
        out = c_double()
        v0 = _vin(v0, self._level_n(level), "v0")
        check(lib().stokes_mg_arnoldi_lmax(self.h, level, _ptr(v0), steps, byref(out), _stream(self.stream)))
        return out.value

    def residual(self, level, b, x, precision=FP64):
        import torch
        n = self._level_n(level)
        b = _vin(b, n, "b")
        x = _vin(x, n, "x")
        r = torch.empty_like(b)
        check(lib().stokes_mg_residual(self.h, level, _ptr(b), _ptr(x), _ptr(r), precision, _stream(self.stream)))
        return r

    def asm(self, level, r, precision=FP64):
        import torch
        r = _vin(r, self._level_n(level), "r")
        z = torch.empty_like(r)
        check(lib().stokes_mg_asm(self.h, level, _ptr(r), _ptr(z), precision, _stream(self.stream)))
        return z

    def transfer(self, level, direction, x, y, precision=FP64):
        """direction 0: y = R_l x (x on level l, y on l + 1); 1: y += P_l x
        (x on l + 1, y on l).  y is written in place."""
        nf, nc = self._level_n(level), self._level_n(level + 1)
        x = _vin(x, nc if direction else nf, "x")
        y = _vout(y, nf if direction else nc, "y")
        check(lib().stokes_mg_transfer(self.h, level, direction, _ptr(x), _ptr(y), precision, _stream(self.stream)))
        return y

    def coarse_solve(self, r):
        import torch
        r = _vin(r, self._nfree[-1], "r")
        x = torch.empty_like(r)
        check(lib().stokes_mg_coarse_solve(self.h, _ptr(r), _ptr(x), _stream(self.stream)))
        return x

    def _level_n(self, level):
        if not 0 <= level < len(self._nfree):
            raise ValueError(f"level {level} outside [0, {len(self._nfree)})")
        return self._nfree[level]

    def prof_enable(self, kind, on=True):
        check(lib().stokes_prof_enable(self.h, kind, int(on)))

    def prof_read(self, kind):
        n, ms = c_longlong(), c_double()
        check(lib().stokes_prof_read(self.h, kind, byref(n), byref(ms)))
        return n.value, ms.value

    def prof_read_one(self, kind, index):
        ms = c_double()
        check(lib().stokes_prof_read_one(self.h, kind, int(index), byref(ms)))
        return ms.value

    def close(self):
        if self.h:
            lib().stokes_mg_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
