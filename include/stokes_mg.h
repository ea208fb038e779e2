/*
 * stokes_mg.h -- C ABI of a GB300 (sm_103a) monolithic ph-multigrid
 * preconditioner for high-order Taylor-Hood and Scott-Vogelius
 * discretisations of stationary Stokes, used inside FGMRES.
 *
 * Method: Voronin, Harper, MacLachlan, Olson, Tuminaro, "Monolithic Multigrid
 * Preconditioners for High-Order Discretizations of Stokes Equations"
 * (arXiv 2407.07253).  Section / equation numbers below refer to it.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, a negative STOKES_E* code on failure; the
 *     message of the last failure on the calling thread is available from
 *     stokes_last_error().  No C++ exception crosses this boundary.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work of a call is ordered on that stream; calls that
 *     return host results synchronise it.
 *   - "device" pointers are CUDA global-memory pointers owned by the caller;
 *     "host" pointers are ordinary CPU memory owned by the caller.  The
 *     library never keeps a caller pointer beyond the call.
 *   - The library owns every buffer it allocates; stokes_mg_destroy frees
 *     them.  A handle is bound to the device that was current at setup.
 *   - DoF order of a level's linear system ("free" vector, length n_free):
 *     free velocity nodes of component 0, then of component 1 (then 2), then
 *     every pressure node.  Dirichlet velocity DoFs are eliminated.  The
 *     coordinates of every free DoF are exported by stokes_mg_level_dofs.
 *   - DoF order of a full field (stokes_solve input/output): velocity of
 *     component 0 at every velocity node (boundary included), component 1,
 *     (component 2); pressure at every pressure node.  Node coordinates are
 *     exported by stokes_mg_nodes.
 */
#ifndef STOKES_MG_H
#define STOKES_MG_H

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define STOKES_OK               0
#define STOKES_EINVAL          -1   /* invalid argument (sizes, family, k, mesh) */
#define STOKES_EOOM            -2   /* device or host allocation failed */
#define STOKES_ESINGULAR       -3   /* zero pivot in a patch or the coarse LU; stats.singular_patch names it */
#define STOKES_ENOTCONVERGED   -4   /* FGMRES reached maxit above tol */
#define STOKES_ENONFINITE      -5   /* NaN/Inf in a residual norm */
#define STOKES_ECUDA           -6   /* a CUDA runtime call failed */
#define STOKES_EUNSUPPORTED    -7   /* valid request outside what this build implements */

/* element families (Sec. 2.1) */
#define STOKES_TH 0   /* Taylor-Hood P_k / P_{k-1}, k >= 2 */
#define STOKES_SV 1   /* Scott-Vogelius P_k / P_{k-1}^disc on an Alfeld-refined mesh, k >= d */

/* p-hierarchy (Sec. 3.2, Fig. 7) */
#define STOKES_HIER_DIRECT   0  /* P_k -> P_2, then h-coarsening */
#define STOKES_HIER_GRADUAL  1  /* Fig. 7 schedule: k<=5 -> 2; k=6,7 -> 4 -> 2; k>=8 -> 5 -> 2 */
#define STOKES_HIER_EXPLICIT 2  /* opts.schedule[0..n_schedule-1] velocity degrees, first = k */
#define STOKES_HIER_HMG      3  /* no p-coarsening: P_k on every mesh (the paper's hMG) */

/* precision of the V-cycle and of the operator inside the lambda_max Arnoldi
 * (FGMRES, the Arnoldi basis, patch LU and coarse LU are FP64 in both) */
#define STOKES_FP64  0
#define STOKES_MIXED 1   /* FP32 SpMV, transfers and patch apply with FP32 accumulation */

typedef struct {
    int dim;               /* 2 (triangles) or 3 (tetrahedra) */
    int n_verts;
    int n_cells;
    const double* verts;   /* host, [n_verts][dim] */
    const int* cells;      /* host, [n_cells][dim+1] vertex indices */
} stokes_mesh;

typedef struct {
    int hierarchy;          /* STOKES_HIER_* */
    int n_schedule;         /* for STOKES_HIER_EXPLICIT */
    int schedule[8];
    int nu_p;               /* Chebyshev degree on the p-levels (Fig. 6b) */
    int nu_h;               /* Chebyshev degree on the hMG levels (Fig. 6a) */
    int n_V;                /* hMG cycles per phMG cycle (Sec. 4.1.1) */
    int eig_steps;          /* Arnoldi steps of the lambda_max estimate */
    unsigned long long eig_seed;  /* SplitMix64 seed of the Arnoldi start vectors */
    double cheb_lo, cheb_hi;      /* Chebyshev interval = [lo, hi] * lambda_max */
    double lmax_override[16];     /* > 0: use instead of the estimate on level i */
    int precision;          /* STOKES_FP64 or STOKES_MIXED */
    int restart;            /* FGMRES restart length (30 in Sec. 4) */
    int maxit;              /* FGMRES iteration limit */
    int use_graph;          /* capture the V-cycle in a CUDA graph (default 1) */
    int host_only;          /* 1: build only the host-side hierarchy (meshes, spaces,
                               CSR operators, transfers, patches) and make no CUDA
                               call; only the info / dofs / nodes / get_csr /
                               get_patches queries are valid on such a handle */
    int prof_mask;          /* bit k set: time kernel class k (see stokes_prof_enable)
                               from the start of setup */
    int patch_solver;       /* exact patch solves (Sec. 3.4), both FP64:
                               0 (default) block inverse of the saddle structure
                                 [L 0 B0^T; 0 L B1^T; B0 B1 0]: SPD L and Schur
                                 complement S = sum B_c L^-1 B_c^T inverted by
                                 Gauss-Jordan without pivoting;
                               1 partial-pivot Gauss-Jordan on the whole patch */
    int batch_tune;         /* batched patch GEMM (stokes_mg_vcycle_batched):
                               1 (default) on first use at a width and mode, time
                               patch-size buckets of every level and keep the
                               fastest split (stokes_batch_plan); 0 one launch
                               per level and kind */
} stokes_mg_opts;

#define STOKES_MAX_LEVELS 16

typedef struct {
    int n_levels;
    int dim, family, k;
    int n_free[STOKES_MAX_LEVELS];
    int degree[STOKES_MAX_LEVELS];        /* velocity degree of each level */
    int level_family[STOKES_MAX_LEVELS];
    int mesh_index[STOKES_MAX_LEVELS];    /* 0 = finest mesh */
    int is_p_level[STOKES_MAX_LEVELS];
    long long nnz[STOKES_MAX_LEVELS];     /* structural nonzeros of K_l (free rows) */
    int n_patches[STOKES_MAX_LEVELS];
    int max_patch[STOKES_MAX_LEVELS];
    long long patch_entries[STOKES_MAX_LEVELS];  /* sum n_i^2 */
    double lmax[STOKES_MAX_LEVELS];       /* lambda_max used by Chebyshev */
    int n_vel_nodes, n_pres_nodes;        /* finest level, full fields */
    int singular_patch;                   /* level*2^24 + patch of the first zero pivot, -1 if none */
    /* setup phase times in ms (host clock for host phases, events for device) */
    double t_mesh_ms, t_assembly_ms, t_upload_ms, t_gather_lu_ms, t_coarse_ms, t_eig_ms, t_graph_ms, t_total_ms;
    long long kernel_launches;            /* launches made by this handle so far */
    /* split of t_assembly_ms (host): spaces + reference tensors, CSR
       matrices, Vanka patches, transfers */
    double t_spaces_ms, t_matrices_ms, t_patches_ms, t_transfers_ms;
    /* busy time of the thread that issues the per-level kernel launches
       while the calling thread assembles (overlapped), and the time the
       calling thread then waited for it */
    double t_launch_thread_ms, t_launch_wait_ms;
    /* uploads issued between levels (t_upload_ms) and after assembly
       (transfers, load operators, t_upload_post_ms) */
    double t_upload_post_ms;
} stokes_mg_stats;

typedef struct stokes_mg* stokes_mg_t;

/* Fill `o` with the defaults: GRADUAL, nu_p = nu_h = n_V = 1, 15 Arnoldi
 * steps, seed 0, interval [0.1, 1.1], precision FP64, restart 30,
 * maxit 1000, use_graph 1. */
void stokes_mg_default_opts(stokes_mg_opts* o);

/* Build the phMG hierarchy and everything a V-cycle needs (Sec. 3, Sec. 4).
 *   coarse           host mesh M_L; the library refines it n_refine times
 *                    (uniform R_u, Fig. 1) and, if barycentric_finest, splits
 *                    the finest mesh by Alfeld (R_b; required for SV).
 *   family, k        STOKES_TH / STOKES_SV and the velocity degree k.
 *   opts             NULL = defaults.
 *   nu_cell          host [cells of the finest mesh] viscosity per cell, or
 *                    NULL for nu = 1 (coarse cells take their children's mean).
 *   stream           device work of setup (gather, LU, eigen-estimate) runs here.
 *   out              receives the handle.
 * Errors: EINVAL (bad mesh/family/k), ESINGULAR (zero pivot; the stats
 * name the patch), EOOM, ECUDA, EUNSUPPORTED (among others: a level whose
 * operator, transfer or patch lists would exceed 2^31 - 1 entries, the
 * range of the 32-bit CSR and list indices). */
int stokes_mg_setup(const stokes_mesh* coarse, int n_refine, int barycentric_finest,
                    int family, int k, const stokes_mg_opts* opts,
                    const double* nu_cell, void* stream, stokes_mg_t* out);

/* z = B_MG r: one phMG V-cycle (Eq. 3.2 on the p-levels, Eq. 3.1 on the
 * h-levels) from a zero initial guess, in the handle's precision.
 * r_dev, z_dev: device, [nrhs][n_free(level 0)] FP64; nrhs >= 1 right-hand
 * sides are processed one after another.  r_dev and z_dev may not alias. */
int stokes_mg_vcycle(stokes_mg_t h, const double* r_dev, double* z_dev, int nrhs, void* stream);

/* FBF(phMG) for Scott-Vogelius (Eq. fbf, Fig. afbf_solver): FGMRES on the SV
 * system of the finest (Alfeld-refined) mesh, right-preconditioned by
 *   P^-1 = [I -A~^-1 B^T; 0 I] diag(A~^-1, S~^-1) [I 0; -B A~^-1 I],
 * with A~^-1 one phMG V-cycle on the velocity block and S~^-1 the inverse of
 * the block-diagonal discontinuous pressure mass matrix.  The velocity block
 * is the vector Laplacian, block diagonal over the components with the same
 * scalar stiffness in each, so A~^-1 is a scalar phMG V-cycle applied to
 * every component; its relaxation is Chebyshev(nu) around one additive
 * Schwarz sweep over ASMStarPC patches (the velocity nodes on the open star of
 * each mesh vertex, Sec. 3.3), with the hierarchy, Chebyshev interval and
 * lambda_max estimate of the monolithic solver.  S~^-1 is
 * -diag_e(nu_e M_p,e^-1): the Schur complement -B A^-1 B^T is negative.
 *   Arguments as stokes_mg_setup (family SV and the barycentric finest mesh
 *   are implied; opts.patch_solver is ignored: Gauss-Jordan).
 * On the returned handle:
 *   stokes_solve / stokes_adjoint_solve   run FGMRES-FBF(phMG) on the Stokes system;
 *   stokes_mg_vcycle                      is A~^-1 on one velocity component
 *                                         ([n_free(level 0)], the scalar level);
 *   stokes_mg_info, stokes_mg_level_dofs, stokes_mg_get_patches, stokes_mg_asm ...
 *                                         describe the scalar velocity levels;
 *   stokes_mg_nodes and the stats' node counts describe the SV Stokes fields;
 *   stokes_grad_viscosity works on the SV level (the finest level is
 *   assembled on the device).
 * Errors: as stokes_mg_setup. */
int stokes_fbf_setup(const stokes_mesh* coarse, int n_refine, int k, const stokes_mg_opts* opts,
                     const double* nu_cell, void* stream, stokes_mg_t* out);

/* z = P^-1 r (Eq. fbf) on an FBF handle.  r_dev, z_dev: device
 * [d * n_free_vel + n_pres] in the Stokes free order (velocity components
 * blocked, then pressure); may not alias.  Errors: EINVAL (not an FBF handle). */
int stokes_fbf_apply(stokes_mg_t h, const double* r_dev, double* z_dev, void* stream);

/* nrhs independent solves K x_c = b_c (c < nrhs <= STOKES_BATCH_MAX) by
 * FGMRES(restart) in lockstep (Sec. 4), every column right-preconditioned
 * by the batched V-cycle of stokes_mg_vcycle_batched (mode STOKES_BATCH_TF32
 * or _3XTF32).  The Krylov arithmetic is FP64 (K applied with its FP64
 * values to all columns at once, classical Gram-Schmidt twice, Givens per
 * column), on the batch interleaved DoF-major; x0 = 0.  Column c counts as
 * converged once its residual estimate is <= tol ||b_c||; the iteration stops
 * when every column has converged (the others keep improving meanwhile).
 *   b_dev, x_dev   device [nrhs][n_free(level 0)] FP64, free-DoF order as
 *                  stokes_mg_fgmres; the pressure part of every b_c must be
 *                  orthogonal to the constants (as stokes_solve's is).
 *   iterations     host out: iterations of the batch; final_relres host
 *                  [nrhs] out or NULL: each column's residual estimate / ||b_c||.
 * Needs a monolithic MIXED handle.  Workspace for (restart + 1) + restart
 * basis vectors of the batch is allocated on first use and kept.
 * Errors: EINVAL, EUNSUPPORTED (patch too large at this width),
 * ENOTCONVERGED, ENONFINITE. */
int stokes_fgmres_batched(stokes_mg_t h, const double* b_dev, double* x_dev, int nrhs, int mode, double tol,
                          int* iterations, double* final_relres, void* stream);

/* Self-test of the bounded mbarrier wait used by the tensor-core kernels
 * (no counterpart in the paper): one CTA waits on a barrier that nothing
 * arrives on, gives up after `polls` polls and returns; *result = 2 then
 * (1 would mean the barrier phase completed, 0 that the kernel never ran).
 * Errors: EINVAL, ECUDA. */
int stokes_selftest_bounded_wait(long long polls, int* result);

/* Measurement utility (no counterpart in the paper): the FP64 pipe's peak on
 * this GPU, the denominator of the roofline of the FP64-bound kernels (the
 * patch inversion).  Launches blocks_per_sm (1..8) CTAs of 256 threads per SM,
 * each thread running 8 independent FP64 FMA chains of `iters` steps, once
 * untimed and once timed with CUDA events on `stream`.
 *   tflops  host out: 2 * 8 * iters * threads / duration, in TFLOP/s;
 *   ms      host out: the timed launch's duration.
 * Allocates one small device buffer (stream-ordered) and synchronises
 * `stream`.  Errors: EINVAL, ECUDA. */
int stokes_probe_fp64_peak(long long iters, int blocks_per_sm, double* tflops, float* ms, void* stream);

/* Discrete adjoint of stokes_solve (differentiation of the solution with
 * respect to the forcing and the cell viscosities).  The paper does not
 * differentiate its solver; this is the standard adjoint of the linear solve
 * of Sec. 2 / Eq. 2.3 with the phMG-preconditioned FGMRES of Sec. 4.
 * For a loss L(u, p) of the outputs of stokes_solve on this handle, with
 *   gu = dL/du   device [dim][n_vel_nodes] (boundary entries are ignored:
 *                the boundary velocity is the Dirichlet data),
 *   gp = dL/dp   device [n_pres_nodes],
 * stokes_adjoint_solve solves K lambda = r (K is symmetric) with the same
 * FGMRES(restart)-phMG to ||r - K lambda|| <= tol ||r||, where r holds gu on
 * the free velocity DoFs and nu * (gp - w (sum gp) / (sum w)) on the
 * pressures (w_j = int psi_j: the transpose of the zero-mean normalisation
 * of p; nu the constant viscosity given to stokes_solve).
 *   lam_u    device [dim][n_vel_nodes] out: lambda's velocity, 0 on the boundary.
 *   lam_p    device [n_pres_nodes] out or NULL: lambda's pressure, zero plain
 *            mean (it is fixed only up to a constant).
 *   grad_f   device [dim][n_vel_nodes] out or NULL: dL/df_nodal = M lam_u / nu,
 *            M the velocity mass matrix (stokes_solve's load is F = M f).
 * Errors: EINVAL, ENOTCONVERGED (outputs hold the last iterate), ENONFINITE. */
int stokes_adjoint_solve(stokes_mg_t h, const double* gu, const double* gp, double nu, double tol, double* lam_u,
                         double* lam_p, double* grad_f, int* iterations, double* final_relres, void* stream);

/* dL/dnu_e = -sum_c lam_u,c[e]^T A_e u_c[e] for every cell e of the finest
 * mesh (in the order of stokes_mg_cell_centroids, which is the order of
 * setup's nu_cell), A_e the cell's unit-viscosity stiffness (Eq. 2.2 with
 * nu = 1 on e), u the velocity returned by stokes_solve (boundary values
 * included) and lam_u from stokes_adjoint_solve; the Dirichlet lifting's
 * dependence on nu is folded in by using the full u.  Valid for a handle
 * whose viscosity is nu_cell (stokes_solve's nu = 1).
 *   u, lam_u  device [dim][n_vel_nodes];  grad  device [n_cells] out.
 * Errors: EINVAL; EUNSUPPORTED when the finest level was assembled on the
 * host (host_only handles). */
int stokes_grad_viscosity(stokes_mg_t h, const double* u, const double* lam_u, double* grad, void* stream);

/* Cells of the finest mesh: *n_cells, and if xyz != NULL their centroids
 * [n_cells][dim] (host) in the library's order, the order of nu_cell and of
 * stokes_grad_viscosity's output. */
int stokes_mg_cell_centroids(stokes_mg_t h, int* n_cells, double* xyz);

/* Z = B_MG R for a batch of right-hand sides in one pass: the same V-cycle
 * as stokes_mg_vcycle (Eq. 3.2 / 3.1, Chebyshev-accelerated ASM relaxation,
 * Sec. 3.3), with the batch interleaved DoF-major on the device so that
 * every sparse matrix is read once per batch and each patch apply
 * W_i K_i^{-1} R_i is a dense (n_i x n_i) x (n_i x m) product on the tensor
 * cores.  The paper applies the preconditioner to one vector at a time; the
 * batch is this library's extension for many independent right-hand sides
 * (block Krylov methods, several load cases).
 *   r_dev, z_dev   device, [nrhs][n_free(level 0)] FP64, as stokes_mg_vcycle;
 *                  may not alias.
 *   nrhs           1 .. STOKES_BATCH_MAX; the batch is padded with zero
 *                  columns to the next width of 8, 16, 32 or 64.
 *   mode           STOKES_BATCH_TF32: TF32 products (about 1e-3 relative);
 *                  STOKES_BATCH_3XTF32: split-TF32 products with FP32
 *                  accuracy (the single-vector MIXED V-cycle to ~1e-5).
 * Needs a MIXED handle (FP32 operators and inverses).  Work buffers of the
 * width are allocated on first use and kept; one CUDA graph per mode and
 * width is captured on first use unless opts.use_graph is 0.
 * Errors: EINVAL (nrhs, mode, an FP64 handle), EUNSUPPORTED (a patch too
 * large for the per-block shared memory at this width), ECUDA. */
#define STOKES_BATCH_MAX    64
#define STOKES_BATCH_TF32   0
#define STOKES_BATCH_3XTF32 1
int stokes_mg_vcycle_batched(stokes_mg_t h, const double* r_dev, double* z_dev, int nrhs, int mode, void* stream);

/* The plan of the batched patch GEMM (the W_i K_i^-1 R_i products of
 * stokes_mg_vcycle_batched) for one relaxed level and mode at the width of
 * the last batched call, set on its first use in that mode.  The level's
 * patches, sorted by size, run as *n_parts launches; launch i covers count[i]
 * patches of sizes lo[i] .. hi[i] and one kind: 1 warp-level MMA, 2 tcgen05
 * tensor cores (TF32 patches of more than 64 DoFs).  warps[i] is the warp
 * kernel's warps per CTA (0: the default for its largest patch).  With
 * opts.batch_tune the buckets and shapes were chosen by timing (part_us[i],
 * microseconds per launch, best of 3), and *single_us is the level as one
 * launch per kind, timed alongside; without it the times are 0.
 *   kind, warps, count, lo, hi, part_us   host [max_parts] out or NULL.
 * Errors: EINVAL (no batched call in this mode at the current width yet,
 * level out of range). */
int stokes_batch_plan(stokes_mg_t h, int mode, int level, int max_parts, int* n_parts, int* kind, int* warps,
                      int* count, int* lo, int* hi, double* part_us, double* single_us);

/* Solve -nu Laplace(u) + grad p = f, div u = 0, u = g on the boundary with
 * FGMRES(restart) right-preconditioned by the V-cycle (Sec. 4), stopped when
 * ||b - K x||_2 <= tol ||b||_2.
 *   f_nodal   device, [dim][n_vel_nodes]: nodal values of f; the load is
 *             F = M f (exact mass-matrix product).
 *   g_nodal   device, [dim][n_vel_nodes] or NULL (homogeneous); only
 *             boundary nodes are read.
 *   nu        constant viscosity > 0 (applied by scaling: the system with
 *             nu = 1 is solved for (u, p/nu)); must be 1 if nu_cell was given.
 *   u         device, [dim][n_vel_nodes] output (boundary values = g).
 *   p         device, [n_pres_nodes] output, zero mean (int p = 0, Sec. 2).
 *   iterations, final_relres   host outputs (may be NULL).
 * Errors: ENOTCONVERGED (outputs hold the last iterate), ENONFINITE. */
int stokes_solve(stokes_mg_t h, const double* f_nodal, const double* g_nodal, double nu,
                 double tol, double* u, double* p, int* iterations, double* final_relres,
                 void* stream);

/* stokes_solve for nrhs independent load cases on one handle (several
 * forcings of the same operator, as a parameter study or a loss summed over
 * forcings): every column's right-hand side is formed as stokes_solve forms
 * it, the columns are solved together by stokes_fgmres_batched (one batched
 * V-cycle per iteration for all of them), and every column's (u, p) is
 * returned as stokes_solve returns it.  The paper solves one load case at a
 * time (Sec. 4); the batch is this library's extension.
 *   f_nodal   device [nrhs][dim][n_vel_nodes].
 *   g_nodal   device [nrhs][dim][n_vel_nodes] or NULL (homogeneous for all).
 *   nrhs      1 .. STOKES_BATCH_MAX;  mode  STOKES_BATCH_TF32 / _3XTF32.
 *   nu, tol   as stokes_solve (the same for every column).
 *   u         device [nrhs][dim][n_vel_nodes] out;  p  device [nrhs][n_pres_nodes] out.
 *   iterations     host out (iterations of the batch);
 *   final_relres   host [nrhs] out or NULL.
 * Needs a monolithic MIXED handle.  Free-DoF buffers of the width are
 * allocated on first use and kept.
 * Errors: EINVAL, EUNSUPPORTED (patch too large at this width),
 * ENOTCONVERGED (outputs hold the last iterate), ENONFINITE. */
int stokes_solve_batched(stokes_mg_t h, const double* f_nodal, const double* g_nodal, int nrhs, int mode, double nu,
                         double tol, double* u, double* p, int* iterations, double* final_relres, void* stream);

/* stokes_adjoint_solve for nrhs loss gradients at once (one per column of a
 * stokes_solve_batched call), solved together by stokes_fgmres_batched.
 *   gu        device [nrhs][dim][n_vel_nodes];  gp  device [nrhs][n_pres_nodes].
 *   lam_u     device [nrhs][dim][n_vel_nodes] out;
 *   lam_p     device [nrhs][n_pres_nodes] out or NULL;
 *   grad_f    device [nrhs][dim][n_vel_nodes] out or NULL.
 *   Other arguments as stokes_solve_batched.
 * Errors: as stokes_solve_batched. */
int stokes_adjoint_solve_batched(stokes_mg_t h, const double* gu, const double* gp, int nrhs, int mode, double nu,
                                 double tol, double* lam_u, double* lam_p, double* grad_f, int* iterations,
                                 double* final_relres, void* stream);

/* grad[e] = -sum_q sum_c lam_u,q,c[e]^T A_e u_q,c[e]: stokes_grad_viscosity
 * summed over nrhs (u, lam_u) pairs, the gradient of a loss summed over the
 * columns of a batched solve, with A_e formed once per cell for all of them.
 *   u, lam_u  device [nrhs][dim][n_vel_nodes];  grad  device [n_cells] out.
 * Errors: as stokes_grad_viscosity. */
int stokes_grad_viscosity_batched(stokes_mg_t h, const double* u, const double* lam_u, int nrhs, double* grad,
                                  void* stream);

/* Sizes and setup statistics (host struct). */
int stokes_mg_info(stokes_mg_t h, stokes_mg_stats* st);

/* Coordinates of the free DoFs of `level` (host outputs, caller-sized):
 *   xyz   [n_free][dim] node coordinates,
 *   comp  [n_free] 0..dim-1 velocity component, dim = pressure,
 *   cell_center [n_free][dim] centroid of the owning cell for discontinuous
 *         pressure DoFs (SV), zeros otherwise (may be NULL). */
int stokes_mg_level_dofs(stokes_mg_t h, int level, double* xyz, int* comp, double* cell_center);

/* Coordinates of the velocity nodes [n_vel_nodes][dim] and pressure nodes
 * [n_pres_nodes][dim] of the finest level (full fields), plus the owning-cell
 * centroid of each pressure node (SV; zeros for TH); host outputs. */
int stokes_mg_nodes(stokes_mg_t h, double* vel_xyz, double* pres_xyz, double* pres_cell_center);

/* ---- per-step entry points (each one step of the hot path) --------------- */

/* which: 0 = K_l, 1 = P_l (coarse l+1 -> fine l), 2 = R_l = P_l^T.
 * Query sizes with row_ptr = NULL: *n_rows, *n_cols, *nnz are returned.
 * Otherwise copies the FP64 CSR into host arrays row_ptr[n_rows+1],
 * col[nnz], val[nnz]. */
int stokes_mg_get_csr(stokes_mg_t h, int level, int which, int* n_rows, int* n_cols,
                      long long* nnz, int* row_ptr, int* col, double* val);

/* Vanka-star patches of a level (Sec. 3.4, Fig. 5): with offsets = NULL
 * returns *n_patches and *n_entries (= sum n_i); otherwise offsets[n+1] and
 * free-DoF indices dofs[sum n_i] (sorted within each patch), host. */
int stokes_mg_get_patches(stokes_mg_t h, int level, int* n_patches, long long* n_entries,
                          int* offsets, int* dofs);

/* a1: dense patch matrices K_i = I_i K I_i^T gathered on the device from the
 * CSR of K_l (Eq. 3.4), written to host out[sum n_i^2], row-major per patch
 * in patch order. */
int stokes_mg_patch_matrices(stokes_mg_t h, int level, double* out, void* stream);

/* a2: explicit inverses K_i^{-1} from the batched partial-pivot
 * Gauss-Jordan kernel (FP64), host out[sum n_i^2], row-major per patch. */
int stokes_mg_patch_inverses(stokes_mg_t h, int level, double* out, void* stream);

/* a3: largest real Ritz value of `steps` Arnoldi steps on M_l^{-1} K_l from
 * the device start vector v0_dev [n_free(level)] (FP64).  The operator is
 * applied in the handle's V-cycle precision (FP32 CSR values and stored
 * inverses for STOKES_MIXED, the smoother the estimate serves); the Krylov
 * basis, its CGS2 orthogonalisation and the Hessenberg matrix are FP64. */
int stokes_mg_arnoldi_lmax(stokes_mg_t h, int level, const double* v0_dev, int steps,
                           double* lmax, void* stream);

/* a4: r = b - K_l x (device vectors, n_free(level)) in `precision`
 * (STOKES_FP64 or STOKES_MIXED = FP32 values/accumulation; inputs and
 * outputs are FP64 and rounded at the boundary). */
int stokes_mg_residual(stokes_mg_t h, int level, const double* b, const double* x, double* r,
                       int precision, void* stream);

/* a5: z = M_l^{-1} r = sum_i I_i^T W_i K_i^{-1} I_i r (Eq. 3.4) with
 * W_i = diag(1/multiplicity), in `precision` (device vectors). */
int stokes_mg_asm(stokes_mg_t h, int level, const double* r, double* z, int precision, void* stream);

/* a6: y = R_l x (restrict, x on level l, y on l+1) if dir = 0;
 *     y += P_l x (prolong-and-add, x on l+1, y on l) if dir = 1. */
int stokes_mg_transfer(stokes_mg_t h, int level, int dir, const double* x, double* y,
                       int precision, void* stream);

/* a7: coarsest-level solve of K_c x = r with the zero-mean pressure
 * constraint (bordered FP64 LU inverse), device vectors. */
int stokes_mg_coarse_solve(stokes_mg_t h, const double* r, double* x, void* stream);

/* FGMRES on the free level-0 system K x = b (device b, x; x0 = 0). */
int stokes_mg_fgmres(stokes_mg_t h, const double* b, double* x, double tol, int* iterations,
                     double* final_relres, void* stream);

/* Kernel timing for measurement: while enabled, the launches of kernel
 * class `kind` (0 = patch apply, 1 = K SpMV, 2 = Gauss-Jordan, 3 = pull
 * scatter, 4 = transfer SpMV) are bracketed with CUDA events on their stream
 * and their total time accumulated (event pairs are read at the next
 * stokes_prof_read).  enable = 0 stops. */
int stokes_prof_enable(stokes_mg_t h, int kind, int enable);
int stokes_prof_read(stokes_mg_t h, int kind, long long* launches, double* total_ms);
/* Duration (ms, CUDA events on the launching stream) of the index-th timed
 * launch of class `kind`, in launch order (0-based; EINVAL if out of range).
 * During setup the patch-inversion launches of the relaxed levels are timed
 * in the order the levels are built (level 0 first). */
int stokes_prof_read_one(stokes_mg_t h, int kind, long long index, double* ms);

/* ---- allocation-free batched inverse ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: applications whose HBM is owned by
 * another allocator (a framework's caching pool that has reserved it, so
 * cudaMalloc would fail or fragment it) and code that must not enter the
 * CUDA allocator at all (cudaFree synchronises the device).
 *
 * Inverts, in place and in FP64, npatch dense row-major matrices packed back
 * to back in `mats` (device, caller-owned): matrix p has size n_p = sizes[p]
 * (host array) and starts at element sum_{q<p} n_q^2.  The algorithm is the
 * batched partial-pivot Gauss-Jordan of stokes_mg_patch_inverses.
 *   sizes[p] in [1, 4096]; npatch <= STOKES_NOALLOC_MAX_PATCHES and
 *   sum of sizes <= STOKES_NOALLOC_MAX_ENTRIES, else STOKES_EINVAL and no
 *   GPU work.
 *   first_singular (host, may be NULL): index of the first patch with a zero
 *   pivot (STOKES_ESINGULAR is returned; its matrix is then not an inverse),
 *   -1 otherwise.
 * Allocates nothing: no cudaMalloc, no cudaFree, no host heap.  Its scratch
 * (offsets, pivot status, pivot workspace of matrices larger than 160) is a
 * fixed array of about 7 MB in this library's device memory, held by every
 * GPU that loads the library until the process exits.  The first call on a
 * device does a one-time set-up: it looks up that array's device address
 * (cudaGetSymbolAddress) with the device current.  Every call shares the
 * one array and it keeps the last call's contents (the pivot status is
 * cleared by each call):
 * GPU work of two calls that overlapped would race on it.  Within one process
 * the entry point prevents that itself: a process-wide lock is held from the
 * staging of the offsets (in static host arrays) until `stream` has drained,
 * so concurrent calls from several host threads, on one device or on
 * several, run one after another.  The call synchronises `stream`.
 * Errors: EINVAL (sizes), ESINGULAR, ECUDA; message from
 * stokes_noalloc_last_error(). */
#define STOKES_NOALLOC_MAX_PATCHES 65536
#define STOKES_NOALLOC_MAX_ENTRIES 524288
int stokes_batched_inverse_noalloc(int npatch, const int* sizes, double* mats, int* first_singular,
                                   void* stream);
const char* stokes_noalloc_last_error(void);

/* Free everything the handle owns (NULL is accepted). */
void stokes_mg_destroy(stokes_mg_t h);

/* Message of the last failure on this thread ("" if none). */
const char* stokes_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_MG_H */
