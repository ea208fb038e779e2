"""Benchmark: FGMRES-phMG time to a 1e-8 relative residual plus setup time,
mixed precision (FP32 V-cycle inside FP64 FGMRES) against FP64, on one GB300.

One step = stokes_mg_setup (mesh refinement, assembly, patch gather, batched
FP64 Gauss-Jordan, coarse LU, Arnoldi estimates, graph capture) + stokes_solve
(load vector, FGMRES(30) preconditioned by the phMG V-cycle, zero-mean
pressure) on the Taylor-Hood P4/P3 64x64 unit-square workload (169,347 DoFs
with boundary, 167,299 free) with seeded U[-1,1] nodal forcing.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME] [--no-cpu-baseline]
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FGMRES-phMG time to 1e-8 residual + setup time, mixed vs FP64 on GB300"
TOL = 1e-8
# relaxation of the main step.  Sec. 4 reports, per run, the fastest of the
# (n_V, nu_p, nu_h) combinations it explored; on the TH P4 problems here that
# is Chebyshev of degree 2 on [0.5, 2.0] lambda_max around one Vanka-star ASM
# sweep, pre and post, with lambda_max from 8 Arnoldi steps (9 / 11 / 12
# iterations on 64^2 / 128^2 / 256^2, where degree 1 on [0.1, 1.1] lambda_max
# from 15 steps takes 20 / 30 / 81).  "v11" is that degree-1 default of the
# library, kept as a comparison.
RELAX = {"v22": dict(nu_p=2, nu_h=2, cheb_lo=0.5, cheb_hi=2.0, eig_steps=8),
         "v11": dict(nu_p=1, nu_h=1, cheb_lo=0.1, cheb_hi=1.1, eig_steps=15)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="th_p4_64x64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single", action="store_true",
                    help="one mixed-precision setup + solve and exit (profiling driver)")
    ap.add_argument("--warmup-single", action="store_true",
                    help="with --single: run --warmup untimed steps before the single step")
    ap.add_argument("--fp64-probe-only", action="store_true",
                    help="only the FP64 pipe peak probe, over launch shapes")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--relaxation", default="v22", choices=sorted(RELAX),
                    help="v22: Chebyshev(2) on [0.5, 2] lmax pre and post; v11: Chebyshev(1) on [0.1, 1.1] lmax")
    ap.add_argument("--no-paper-scale", action="store_true",
                    help="skip the 2.7 M DoF TH P4 256 x 256 measurement")
    ap.add_argument("--batched-workload", default="th_p3_cube16",
                    help="workload of the batched multi-RHS V-cycle measurement")
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--batch-tune", type=int, default=1, choices=[0, 1],
                    help="batched section: 1 autotuned patch-size buckets, 0 one launch per level and kind")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched V-cycle measurement (profiling driver)")
    ap.add_argument("--adjoint-workload", default="th_p3_128x128_nu",
                    help="workload of the adjoint (gradient) measurement")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-nrhs", type=int, default=32,
                    help="forcings of the batched forward + backward of the adjoint workload")
    ap.add_argument("--fbf-workload", default="sv_p4_disk",
                    help="Scott-Vogelius workload of the FBF(phMG) versus monolithic phMG measurement")
    ap.add_argument("--no-fbf", action="store_true")
    ap.add_argument("--no-highk", action="store_true", help="skip the direct-versus-gradual P6 / P8 measurement")
    ap.add_argument("--highk-only", action="store_true", help="only the high-order measurement")
    ap.add_argument("--fbf-only", action="store_true", help="only the FBF measurement (profiling driver)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the adjoint measurement (profiling driver)")
    return ap.parse_args()


def max_over_ranks(value, pg, device):
    """The largest per-replica value over all ranks (a step is as slow as the
    slowest replica); pg is torch.distributed or None for one process."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- oracle leg
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import multigrid as mg
w = W.workload({name!r})
t0 = time.perf_counter()
h = mg.Hierarchy(w.verts, w.cells, w.n_refine, w.family, w.schedule, barycentric=w.barycentric,
                 opts=mg.Options(**{relax!r}))
t1 = time.perf_counter()
D = h.levels[0].disc
f = W.nodal_forcing(D.V.n, D.d, w.seed)
full, its, hist, b, x = mg.solve(h, f, None, tol={tol!r})
t2 = time.perf_counter()
if {save!r}:
    # untimed: the same forcing solved to a relative residual of {tight!r}
    # (the discrete solution to rounding), and the owner-cell centroid of
    # every pressure node (discontinuous pressures share coordinates)
    full_tight = mg.solve(h, f, None, tol={tight!r})[0]
    cells = np.asarray(D.cells)
    cent = D.verts[cells].mean(axis=1)
    owner = np.zeros(D.Q.n, dtype=np.int64)
    for ci in range(len(cells)):
        owner[D.Q.cell_nodes[ci]] = ci
    pc = cent[owner] if not D.Q.continuous else np.zeros_like(D.Q.coords)
    np.savez({save!r}, full=full, full_tight=full_tight, vx=D.V.coords, px=D.Q.coords, pc=pc)
print(json.dumps(dict(setup_s=t1 - t0, solve_s=t2 - t1, its=its, relres=hist[-1])))
"""
TIGHT = 1e-14         # the oracle's tight solve (its pinned route to the discrete solution)
TIGHT_LIB = 1e-13     # the library's FP64 solve compared with it


def run_oracle(name, relax, timeout=900, save=None, threads=1):
    """The FP64 CPU oracle, as it stands, in a fresh process whose BLAS uses
    `threads` threads, with the relaxation parameters of the GPU step (its
    solutions and node coordinates written to `save`, an .npz path, when
    given; outside the timed part)."""
    t = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, tol=TOL, relax=RELAX[relax], save=save, tight=TIGHT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=timeout, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def node_perm(lib_xyz, ora_xyz, lib_center=None, ora_center=None):
    """perm such that library node perm[i] is oracle node i, matched by
    coordinates rounded to 1e-9 and, for discontinuous spaces (several nodes
    at one position), the owning cell's centroid.  Raises if a key is not
    unique or has no partner."""
    import numpy as np

    def key(x, c):
        a = np.round(np.asarray(x) * 1e9).astype(np.int64)
        if c is not None:
            a = np.concatenate([a, np.round(np.asarray(c) * 1e9).astype(np.int64)], axis=1)
        return [tuple(r) for r in a.tolist()]

    kl, ko = key(lib_xyz, lib_center), key(ora_xyz, ora_center)
    where = {k: i for i, k in enumerate(kl)}
    if len(where) != len(kl) or len(set(ko)) != len(ko) or len(kl) != len(ko):
        raise ValueError("node keys are not unique: pass the owner-cell centroids of discontinuous nodes")
    return np.array([where[k] for k in ko])


def oracle_error(P, W, w, npz, solve):
    """Relative max-norm differences between the GPU solutions and the
    oracle's for the oracle's forcing: the seeded nodal values in the
    oracle's node order, moved to the library's nodes by their coordinates
    (an input permutation; the timed steps draw the same generator in the
    library's order).
      mixed, fp64   library solved to TOL against the oracle solved to TOL
                    (they differ by about TOL times the condition number);
      fp64_tight    library FP64 solved to TIGHT_LIB against the oracle solved
                    to TIGHT, i.e. both at the discrete solution: the accuracy
                    target of 1e-10 relative for u and the zero-mean p.
    solve(precision, f, tol) returns (u, p) of the library as numpy arrays;
    pressures are both zero-mean."""
    import numpy as np

    z = np.load(npz)
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                       hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, host_only=1)
    vx, px, pc = probe.nodes()
    probe.close()
    disc = bool(np.abs(z["pc"]).max() > 0)
    pv = node_perm(vx, z["vx"])
    pq = node_perm(px, z["px"], pc if disc else None, z["pc"] if disc else None)
    d, nV = w.verts.shape[1], len(z["vx"])
    f_lib = np.empty((d, nV))
    f_lib[:, pv] = W.nodal_forcing(nV, d, w.seed)
    out = {}
    for tag, prec, tol, ref in (("mixed", P.MIXED, TOL, "full"), ("fp64", P.FP64, TOL, "full"),
                                ("fp64_tight", P.FP64, TIGHT_LIB, "full_tight")):
        u_o = z[ref][:d * nV].reshape(d, nV)
        p_o = z[ref][d * nV:]
        u, p = solve(prec, f_lib, tol)
        U = u.reshape(d, -1)[:, pv]
        out[tag] = {"u_rel": float(np.abs(U - u_o).max() / np.abs(u_o).max()),
                    "p_rel": float(np.abs(p[pq] - p_o).max() / np.abs(p_o).max()), "tol": tol}
    out["fp64_tight"]["oracle_tol"] = TIGHT
    out["note"] = (f"max-norm differences, relative to the oracle's max. mixed and fp64: both sides stop at {TOL} "
                   "relative residual, so they differ by about that tolerance times the condition number. "
                   f"fp64_tight: the library's FP64 path at {TIGHT_LIB} against the oracle at {TIGHT} (target 1e-10)")
    return out


def relax_text(name):
    r = RELAX[name]
    return (f"V({r['nu_p']},{r['nu_h']}): Chebyshev degree {r['nu_p']} (p-levels) / {r['nu_h']} (h-levels) on "
            f"[{r['cheb_lo']}, {r['cheb_hi']}] x lambda_max ({r['eig_steps']} Arnoldi steps) around one "
            "Vanka-star ASM sweep, pre and post")


def step_config(a, w, world):
    """The workload of one step, identical in both arms."""
    return {"workload": a.workload, "family": "TH" if w.family == 0 else "SV", "k": w.k,
            "schedule": list(w.schedule), "tol": TOL, "relaxation": relax_text(a.relaxation),
            "parallelism": f"replicas{world}"}


def reference_arm(a):
    import workloads as W

    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = W.workload(a.workload)
    runs = []
    for _ in range(max(1, a.steps)):
        runs.append(run_oracle(a.workload, a.relaxation))
    ms = [1e3 * (r["setup_s"] + r["solve_s"]) for r in runs]
    value = sum(ms) / len(ms)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": value, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(a, w, world),
        "precision": "FP64 throughout (numpy/scipy)",
        "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "host_cores": os.cpu_count() or 1,
                         "kind": "oracle",
                         "sample": f"full setup + FGMRES solve of {a.workload} per step, {relax_text(a.relaxation)}, "
                                   "single-threaded numpy/scipy",
                         "iterations": runs[0]["its"]},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"stokes_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def batched_section(a, P, W, dev, stream, flush, hbm):
    """Batched V-cycle (m right-hand sides interleaved, patch apply as a
    per-patch GEMM on the tensor cores) on its own workload: time per
    V-cycle for the whole batch in both modes against m single-RHS mixed
    V-cycles, the end-to-end call with host buffers, and the roofline of
    level 0's TF32 patch GEMM (one launch, CUDA events on its stream)."""
    import numpy as np
    import torch

    w = W.workload(a.batched_workload)
    m = a.nrhs

    def make(prof_mask=0):
        return P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                          hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, precision=P.MIXED,
                          stream=stream.cuda_stream, prof_mask=prof_mask, batch_tune=a.batch_tune)

    h = make()
    n = h.info()["n_free"][0]
    R_host = torch.tensor(np.random.default_rng(w.seed + 1).standard_normal((m, n))).pin_memory()
    Z_host = torch.empty_like(R_host).pin_memory()
    R = R_host.to(dev)
    Z = torch.empty_like(R)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        out = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return sorted(out)[len(out) // 2]

    reps = max(5, a.steps)
    l0 = h.info()["kernel_launches"]
    h.vcycle_batched(R, P.BATCH_TF32, out=Z)
    torch.cuda.synchronize(dev)
    launches = h.info()["kernel_launches"] - l0
    tf32_ms = timed(lambda: h.vcycle_batched(R, P.BATCH_TF32, out=Z), reps)
    x3_ms = timed(lambda: h.vcycle_batched(R, P.BATCH_3XTF32, out=Z), reps)
    k1 = min(8, m)
    single_ms = timed(lambda: h.vcycle(R[:k1], out=Z[:k1]), reps) / k1

    def e2e():
        Rd = R_host.to(dev, non_blocking=True)
        Zd = h.vcycle_batched(Rd, P.BATCH_TF32)
        Z_host.copy_(Zd, non_blocking=True)
    e2e_ms = timed(e2e, reps)
    # the whole solve: m FGMRES-phMG solves to TOL in lockstep (TF32 batched
    # V-cycle, FP64 Krylov arithmetic) against one single-RHS solve per RHS
    i0 = h.info()
    Bq = R.clone()
    pm0 = i0["n_free"][0] - i0["n_pres_nodes"]
    Bq[:, pm0:] -= Bq[:, pm0:].mean(dim=1, keepdim=True)        # consistent pressure parts
    solve_out = {}

    def bsolve():
        solve_out["r"] = h.fgmres_batched(Bq, P.BATCH_TF32, tol=TOL)
    bsolve_ms = timed(bsolve, 3)
    _, bits, brel = solve_out["r"]

    def ssolve():
        solve_out["s"] = h.fgmres(Bq[0].clone(), tol=TOL)
    ssolve_ms = timed(ssolve, 3)
    h.close()

    # level-0 TF32 patch GEMM launches, CUDA events recorded by the library
    # on the launching stream (eager path)
    hp = make(1 << P._binding.PROF_PATCH)
    npatch_levels = hp.info()["n_levels"] - 1
    off, _ = hp.patches(0)
    n_i = np.diff(off).astype(np.float64)
    ld_i = np.floor((n_i + 3) / 4) * 4
    for _ in range(3):
        hp.vcycle_batched(R, P.BATCH_TF32, out=Z)
    torch.cuda.synchronize(dev)
    plan0, single0 = hp.batch_plan(0, P.BATCH_TF32)
    plans = {}
    for mode_name, mode in (("tf32", P.BATCH_TF32), ("3xtf32", P.BATCH_3XTF32)):
        hp.vcycle_batched(R, mode, out=Z)
        plans[mode_name] = []
        for li in range(npatch_levels):
            parts, single = hp.batch_plan(li, mode)
            plans[mode_name].append({"launches": [[pt["lo"], pt["hi"], pt["count"], "tc" if pt["kind"] == 2 else "warp",
                                                   pt["warps"]] for pt in parts],
                                     "tuned_us": sum(pt["us"] for pt in parts), "one_per_kind_us": single})
    per = []
    for _ in range(reps):
        k0 = hp.prof_read(P._binding.PROF_PATCH)[0]
        flush.fill_(1.0)
        hp.vcycle_batched(R, P.BATCH_TF32, out=Z)
        torch.cuda.synchronize(dev)
        k1_ = hp.prof_read(P._binding.PROF_PATCH)[0]
        ms = [hp.prof_read_one(P._binding.PROF_PATCH, i) for i in range(k0, k1_)]
        per.append(sum(ms[:len(plan0)]))  # the cycle's first patch launches: level 0, pre-smoothing
    hp.close()
    gemm_ms = sorted(per)[len(per) // 2]
    # algorithmic bytes: FP32 inverses once + Yb written (n_i x m) + X read once
    gemm_bytes = 4.0 * float((n_i * ld_i).sum()) + 4.0 * m * float(n_i.sum()) + 4.0 * m * n
    gemm_flop = 2.0 * m * float((n_i * n_i).sum())
    gemm_gbs = gemm_bytes / (gemm_ms * 1e-3) / 1e9
    # DRAM traffic per launch: the last ncu capture of the tensor-core launch
    # (level 0 of th_p3_cube8 at 64 right-hand sides, batch_tune 0:
    # dram__bytes_read.sum + dram__bytes_write.sum = 440.98 + 43.14 MB
    # against 471.24 MB of algorithmic bytes) predates the 3xTF32 split of the
    # kernel, so no traffic is reported for the current kernel
    traffic = None
    traffic_src = ("not re-captured since the kernel gained its 3xTF32 split; the TF32 launch measured "
                   "484.1 MB for 471.2 MB algorithmic (1.03x) on th_p3_cube8 before that change")
    return {
        "workload": a.batched_workload, "nrhs": m, "n_free": n, "relaxed_levels": npatch_levels,
        "vcycle_ms": {"tf32": tf32_ms, "3xtf32": x3_ms, "single_rhs_mixed_per_rhs": single_ms},
        "rhs_per_s": {"tf32": 1e3 * m / tf32_ms, "3xtf32": 1e3 * m / x3_ms, "single_rhs": 1e3 / single_ms},
        "speedup_vs_single_rhs": {"tf32": single_ms * m / tf32_ms, "3xtf32": single_ms * m / x3_ms},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(R_host.numel() * 8),
                "d2h_bytes_per_step": int(Z_host.numel() * 8)},
        "gpu_launches_per_vcycle": launches,
        "solve": {"batched_fgmres_ms": bsolve_ms, "iterations": bits, "max_relres": float(max(brel)),
                  "single_rhs_fgmres_ms": ssolve_ms, "single_rhs_iterations": solve_out["s"][1],
                  "rhs_per_s": 1e3 * m / bsolve_ms, "speedup_vs_single_rhs": ssolve_ms * m / bsolve_ms,
                  "note": f"{m} seeded right-hand sides (pressure parts mean-free), tol {TOL}, TF32 batched "
                          "V-cycle preconditioner, FP64 Krylov; single-RHS = stokes_mg_fgmres on the first"},
        "patch_gemm_plans": plans,
        "roofline": {"kernel": f"k_patch_gemm (tcgen05 TF32 and warp MMA), level 0, its {len(plan0)} tuned launches "
                               f"(one launch per kind: {single0:.1f} us)", "bound": "hbm",
                     "achieved": gemm_gbs, "peak": hbm, "unit": "GB/s", "frac": gemm_gbs / hbm,
                     "bytes_per_launch": gemm_bytes, "us_per_launch": 1e3 * gemm_ms,
                     "tf32_tflops": gemm_flop / (gemm_ms * 1e-3) / 1e12,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "l2": "flushed (256 MB write) before every timed V-cycle",
    }


def buckets_section(a, P, W, dev, stream, flush, m=64):
    """The batched V-cycle on the Scott-Vogelius disk, whose level-0 patches
    come in several sizes (92 DoFs at the Alfeld centres, 130-482 at the
    macro vertices): m right-hand sides, each mode, with the autotuned
    patch-size buckets and with one launch per level and kind
    (batch_tune = 0); CUDA events, L2 flushed, median of the timed runs."""
    import numpy as np
    import torch

    w = W.workload(a.fbf_workload)
    out = {"workload": a.fbf_workload, "nrhs": m}
    hs = {}
    for tag, tune in (("tuned", 1), ("one_per_kind", 0)):
        hs[tag] = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                             hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, precision=P.MIXED,
                             stream=stream.cuda_stream, batch_tune=tune)
    n = hs["tuned"].info()["n_free"][0]
    R = torch.tensor(np.random.default_rng(w.seed + 3).standard_normal((m, n)), device=dev)
    Z = torch.empty_like(R)
    for mode_name, mode in (("tf32", P.BATCH_TF32), ("3xtf32", P.BATCH_3XTF32)):
        res = {}
        for tag, h in hs.items():
            for _ in range(3):
                h.vcycle_batched(R, mode, out=Z)
            ts = []
            for _ in range(max(5, a.steps)):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.vcycle_batched(R, mode, out=Z)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            res[tag + "_ms"] = sorted(ts)[len(ts) // 2]
        parts, single = hs["tuned"].batch_plan(0, mode)
        res["level0_launches"] = [[pt["lo"], pt["hi"], pt["count"], "tc" if pt["kind"] == 2 else "warp", pt["warps"]]
                                  for pt in parts]
        res["level0_tuned_us"] = sum(pt["us"] for pt in parts)
        res["level0_one_per_kind_us"] = single
        res["speedup"] = res["one_per_kind_ms"] / res["tuned_ms"]
        out[mode_name] = res
    for h in hs.values():
        h.close()
    return out


def adjoint_section(a, P, W, dev, stream, flush):
    """Forward (setup with per-cell viscosity + solve) and backward (adjoint
    FGMRES-phMG solve, dL/df and dL/dnu kernels) for one seeded forcing and
    one seeded loss gradient L = gu . u + gp . p, CUDA events on the stream,
    L2 flushed before each phase; then the workload's batch of seeded
    forcings forward and backward at once (adjoint_batched), against the same
    number of single-forcing forward + backward passes."""
    import numpy as np
    import torch

    w = W.workload(a.adjoint_workload)
    kw = dict(barycentric=w.barycentric, hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, precision=P.MIXED,
              stream=stream.cuda_stream)
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                       hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, host_only=1)
    nc = probe.n_cells()
    i0 = probe.info()
    probe.close()
    nV, nQ, d = i0["n_vel_nodes"], i0["n_pres_nodes"], w.verts.shape[1]
    nu = W.cell_viscosity(nc, w.seed)
    rng = np.random.default_rng(w.seed + 7)
    f = torch.tensor(W.nodal_forcing(nV, d, w.seed).reshape(-1), device=dev)
    gu = torch.tensor(rng.standard_normal((d, nV)), device=dev)
    gp = torch.tensor(rng.standard_normal(nQ), device=dev)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def run():
        flush.fill_(1.0)
        e0 = ev()
        h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, nu_cell=nu, **kw)
        u, p, its, rel = h.solve(f, tol=TOL)
        e1 = ev()
        e1.synchronize()
        flush.fill_(1.0)
        e2 = ev()
        lam_u, _, gf, aits, arel = h.adjoint(gu, gp, tol=TOL)
        e3 = ev()
        gnu = h.grad_viscosity(u, lam_u)
        e4 = ev()
        e4.synchronize()
        out = dict(forward=e0.elapsed_time(e1), adjoint_solve=e2.elapsed_time(e3), grad_nu=e3.elapsed_time(e4),
                   its=its, adjoint_its=aits, adjoint_relres=arel, gnu_norm=float(gnu.norm()),
                   launches=h.info()["kernel_launches"])
        h.close()
        return out

    run()                                   # warm-up
    reps = [run() for _ in range(max(3, min(a.steps, 5)))]
    med = {k: sorted(r[k] for r in reps)[len(reps) // 2] for k in ("forward", "adjoint_solve", "grad_nu")}
    batched = adjoint_batched(a, P, W, w, nu, nV, d, dev, stream, flush, kw)
    batched["sequential_single_ms"] = a.adjoint_nrhs * (med["forward"] + med["adjoint_solve"] + med["grad_nu"])
    batched["speedup_vs_sequential_single"] = batched["sequential_single_ms"] / batched["total_ms"]
    return {
        "batched": batched,
        "workload": a.adjoint_workload, "n_cells": nc, "n_free": i0["n_free"][0],
        "forward_ms": med["forward"], "backward_ms": med["adjoint_solve"] + med["grad_nu"],
        "adjoint_solve_ms": med["adjoint_solve"], "grad_nu_kernel_ms": med["grad_nu"],
        "backward_over_forward": (med["adjoint_solve"] + med["grad_nu"]) / med["forward"],
        "fgmres_its": reps[-1]["its"], "adjoint_fgmres_its": reps[-1]["adjoint_its"],
        "adjoint_relres": reps[-1]["adjoint_relres"], "tol": TOL,
        "loss": "L = gu . u + gp . p, gu and gp seeded N(0, 1); f seeded U[-1, 1] nodal; nu_e = exp(N(0, 1/4))",
        "l2": "flushed (256 MB write) before the forward and before the backward",
    }


def adjoint_batched(a, P, W, w, nu, nV, d, dev, stream, flush, kw):
    """The adjoint workload's nrhs seeded forcings through the batched
    autograd wrapper: forward = setup with nu_cell + stokes_solve_batched,
    backward (L = sum_q 0.5 ||u_q - u_target||^2, u_target seeded U[-1, 1]
    nodal) = stokes_adjoint_solve_batched + stokes_grad_viscosity_batched.
    CUDA events on the stream, L2 flushed before each phase, median of the
    timed repetitions after one warm-up."""
    import numpy as np
    import torch
    from paper_2407_07253_gb300 import autograd as PA

    nb = a.adjoint_nrhs
    F0 = torch.tensor(np.stack([W.nodal_forcing(nV, d, w.seed + 100 + q) for q in range(nb)]), device=dev)
    ut = torch.tensor(np.random.default_rng(w.seed + 9).uniform(-1.0, 1.0, (d, nV)), device=dev)
    kwb = {k: v for k, v in kw.items() if k != "precision"}

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def run():
        F = F0.clone().requires_grad_(True)
        nu_t = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
        flush.fill_(1.0)
        e0 = ev()
        U, Pp = PA.solve_batched(w.verts, w.cells, w.n_refine, w.family, w.k, F, nu_t, tol=TOL,
                                 mode=P.BATCH_3XTF32, precision=P.MIXED, **kwb)
        e1 = ev()
        L = 0.5 * ((U - ut) ** 2).sum()
        e1.synchronize()
        flush.fill_(1.0)
        e2 = ev()
        L.backward()
        e3 = ev()
        e3.synchronize()
        return dict(forward=e0.elapsed_time(e1), backward=e2.elapsed_time(e3),
                    gf_norm=float(F.grad.norm()), gnu_norm=float(nu_t.grad.norm()))

    run()
    reps = [run() for _ in range(max(3, min(a.steps, 5)))]
    fw = sorted(r["forward"] for r in reps)[len(reps) // 2]
    bw = sorted(r["backward"] for r in reps)[len(reps) // 2]
    return {"nrhs": nb, "forward_ms": fw, "backward_ms": bw, "total_ms": fw + bw,
            "forcings_per_s": 1e3 * nb / (fw + bw), "mode": "3xtf32 batched V-cycle, FP64 batched FGMRES",
            "loss": "sum_q 0.5 ||u_q - u_target||^2, f_q seeded U[-1, 1] nodal (seeds seed+100+q)",
            "grad_norms": {"f": reps[-1]["gf_norm"], "nu": reps[-1]["gnu_norm"]}}


def paper_scale_section(P, W, dev, stream, flush, reps=3):
    """TH P4/P3 on the 256 x 256 mesh (2.7 M free DoFs; the size of the
    paper's 2D Taylor-Hood runs): one step (setup + mixed-precision solve to
    TOL, L2 flushed, CUDA events) with each relaxation, median of `reps`
    after one warm-up."""
    import torch

    w = W.workload("th_p4_256x256")
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT,
                       schedule=w.schedule, host_only=1)
    i0 = probe.info()
    probe.close()
    f = torch.tensor(W.nodal_forcing(i0["n_vel_nodes"], w.verts.shape[1], w.seed).reshape(-1), device=dev)
    res = {"workload": "th_p4_256x256", "n_free": int(i0["n_free"][0]), "levels": int(i0["n_levels"])}
    for name in ("v22", "v11"):
        runs = []
        for r in range(reps + 1):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT,
                           schedule=w.schedule, precision=P.MIXED, stream=stream.cuda_stream, **RELAX[name])
            st = h.info()
            u, p, its, rel = h.solve(f, tol=TOL)
            e1.record(stream)
            e1.synchronize()
            if r:
                runs.append((e0.elapsed_time(e1), st["t_total_ms"], its, rel))
            h.close()
        runs.sort()
        ms, setup, its, rel = runs[len(runs) // 2]
        res[name] = {"step_ms": ms, "setup_ms": setup, "iterations": its, "relres": rel}
    res["v11_over_v22"] = res["v11"]["step_ms"] / res["v22"]["step_ms"]
    return res


def highk_section(a, P, W, dev, stream, flush, reps=3):
    """High order (Fig. 7, Sec. 4.1.1): TH P6/P5 and P8/P7 on the 32 x 32
    square, one step (setup + mixed-precision solve to TOL, L2 flushed, CUDA
    events) with direct p-coarsening k -> 2 and with the gradual schedule of
    Fig. 7, median of `reps` after one warm-up, with the bench relaxation."""
    import torch

    res = {"relaxation": relax_text(a.relaxation)}
    for name in ("th_p6_32x32", "th_p8_32x32"):
        w = W.workload(name)
        probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT,
                           schedule=w.schedule, host_only=1)
        i0 = probe.info()
        probe.close()
        f = torch.tensor(W.nodal_forcing(i0["n_vel_nodes"], w.verts.shape[1], w.seed).reshape(-1), device=dev)
        row = {"n_free": int(i0["n_free"][0]), "max_patch": int(i0["max_patch"][0])}
        for hier, sched in (("direct", [w.k, 2]), ("gradual", list(w.schedule))):
            runs = []
            try:
                for r in range(reps + 1):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT,
                                   schedule=sched, precision=P.MIXED, stream=stream.cuda_stream,
                                   **RELAX[a.relaxation])
                    st = h.info()
                    u, p, its, rel = h.solve(f, tol=TOL)
                    e1.record(stream)
                    e1.synchronize()
                    if r:
                        runs.append((e0.elapsed_time(e1), st["t_total_ms"], its, rel))
                    h.close()
                runs.sort()
                ms, setup, its, rel = runs[len(runs) // 2]
                row[hier] = {"schedule": sched, "step_ms": ms, "setup_ms": setup, "iterations": its, "relres": rel}
            except Exception as e:  # noqa: BLE001
                row[hier] = {"schedule": sched, "error": str(e)[:200]}
        res[name] = row
    return res


def fbf_section(a, P, W, dev, stream, flush):
    """Scott-Vogelius: one step (setup + solve to TOL, mixed precision, L2
    flushed, CUDA events) with FBF(phMG) (Eq. fbf) and with the monolithic
    phMG, on the same workload and forcing; median of the timed steps after
    one warm-up each."""
    import numpy as np
    import torch

    w = W.workload(a.fbf_workload)
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                       hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, host_only=1)
    i0 = probe.info()
    probe.close()
    d = w.verts.shape[1]
    f = torch.tensor(W.nodal_forcing(i0["n_vel_nodes"], d, w.seed).reshape(-1), device=dev)

    def step(fbf):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                       hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, precision=P.MIXED, stream=stream.cuda_stream,
                       fbf=fbf)
        st = h.info()
        u, p, its, rel = h.solve(f, tol=TOL)
        e1.record(stream)
        e1.synchronize()
        out = dict(ms=e0.elapsed_time(e1), setup_ms=st["t_total_ms"], its=its, rel=rel,
                   launches=h.info()["kernel_launches"], u=u.norm().item(), levels=st["n_levels"],
                   n_free0=st["n_free"][0])
        h.close()
        return out

    res = {}
    for name, fb in (("fbf_phmg", True), ("monolithic_phmg", False)):
        step(fb)
        runs = [step(fb) for _ in range(max(3, min(a.steps, 5)))]
        ms = sorted(r["ms"] for r in runs)[len(runs) // 2]
        res[name] = {"step_ms": ms, "setup_ms": sorted(r["setup_ms"] for r in runs)[len(runs) // 2],
                     "iterations": runs[-1]["its"], "relres": runs[-1]["rel"],
                     "levels": runs[-1]["levels"], "n_free_level0": runs[-1]["n_free0"],
                     "gpu_launches": runs[-1]["launches"]}
    res["workload"] = a.fbf_workload
    res["n_free_stokes"] = int(i0["n_free"][0])
    res["monolithic_over_fbf"] = res["monolithic_phmg"]["step_ms"] / res["fbf_phmg"]["step_ms"]
    res["note"] = ("FBF's level-0 n_free is the scalar velocity level; both solve the same SV system to "
                   f"{TOL} (mixed precision V-cycles, FP64 FGMRES)")
    return res


def main():
    a = parse()
    if a.impl == "reference":
        reference_arm(a)
        return
    import numpy as np
    import torch

    import paper_2407_07253_gb300 as P
    import workloads as W

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    P.lib()
    w = W.workload(a.workload)
    stream = torch.cuda.current_stream(dev)

    def make(precision, prof_mask=0, relax=a.relaxation):
        return P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                          hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, precision=precision,
                          stream=stream.cuda_stream, prof_mask=prof_mask, **RELAX[relax])

    # forcing in the library's node order (seeded U[-1,1] nodal values)
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                       hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, host_only=1)
    info0 = probe.info()
    probe.close()
    nV, nQ, d = info0["n_vel_nodes"], info0["n_pres_nodes"], w.verts.shape[1]
    f_host = torch.tensor(W.nodal_forcing(nV, d, w.seed).reshape(-1)).pin_memory()
    f_dev = f_host.to(dev)
    u_dev = torch.empty(d * nV, dtype=torch.float64, device=dev)
    p_dev = torch.empty(nQ, dtype=torch.float64, device=dev)
    u_host = torch.empty(d * nV, dtype=torch.float64).pin_memory()
    p_host = torch.empty(nQ, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    def one_step(precision, e2e=False, prof=None, relax=a.relaxation):
        flush.fill_(1.0)                      # L2 flush between steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = make(precision, sum(1 << k for k in (prof or [])), relax)
        if e2e:
            f = f_host.to(dev, non_blocking=True)
        else:
            f = f_dev
        u, p, its, rel = h.solve(f, tol=TOL, u=u_dev, p=p_dev)
        if e2e:
            u_host.copy_(u, non_blocking=True)
            p_host.copy_(p, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        st = h.info()
        pr = {k: h.prof_read(k) for k in (prof or [])}
        if P._binding.PROF_GJ in (prof or []) and pr[P._binding.PROF_GJ][0] > 0:
            pr["gj0"] = h.prof_read_one(P._binding.PROF_GJ, 0)     # level 0's inversion launch
        h.close()
        return e0.elapsed_time(e1), its, rel, st, pr

    if a.fbf_only:
        print(json.dumps(fbf_section(a, P, W, dev, stream, flush)))
        return
    if a.adjoint_only:
        print(json.dumps(adjoint_section(a, P, W, dev, stream, flush)))
        return
    if a.fp64_probe_only:
        out = {}
        P._binding.probe_fp64_peak(1 << 12, 2, stream=stream.cuda_stream)
        for bps in (1, 2, 4, 8):
            r = sorted(P._binding.probe_fp64_peak(1 << 17, bps, stream=stream.cuda_stream)[0] for _ in range(3))
            out[f"ctas_per_sm_{bps}"] = r[1]
        print(json.dumps({"fp64_probe_tflops": out}))
        return
    if a.highk_only:
        print(json.dumps(highk_section(a, P, W, dev, stream, flush)))
        return
    if a.batched_only:
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        hbm_only = json.load(open(peaks_path)).get("hbm_gbs", 6800.0) if os.path.exists(peaks_path) else 6800.0
        res = batched_section(a, P, W, dev, stream, flush, hbm_only)
        res["buckets"] = buckets_section(a, P, W, dev, stream, flush)
        print(json.dumps(res))
        return
    if a.single:
        # a.warmup untimed steps first (STOKES_TRACE=1 then also traces warm setups)
        for _ in range(a.warmup if a.warmup_single else 0):
            one_step(P.MIXED if a.precision == "mixed" else P.FP64)
        ms, its, rel, st, _ = one_step(P.MIXED if a.precision == "mixed" else P.FP64)
        torch.cuda.synchronize(dev)
        print(json.dumps({"single_step_ms": ms, "iterations": its, "relres": rel,
                          "setup_ms": st["t_total_ms"], "launches": st["kernel_launches"]}))
        return
    # warm-up
    for _ in range(a.warmup):
        one_step(P.MIXED)
    barrier()
    # timed region: mixed precision, inputs resident in HBM
    times, its_l, launches, gj_prof, gj0 = [], [], 0, [0, 0.0], []
    stats = None
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(a.steps):
            ms, its, rel, st, pr = one_step(P.MIXED, prof=[P._binding.PROF_GJ])
            times.append(ms)
            its_l.append(its)
            launches += st["kernel_launches"]
            gj_prof[0] += pr[P._binding.PROF_GJ][0]
            gj_prof[1] += pr[P._binding.PROF_GJ][1]
            gj0.append(pr.get("gj0", 0.0))
            stats = st
        barrier()
        wall = time.perf_counter() - t0
    ms_local = sum(times) / len(times)
    ms_max = max_over_ranks(ms_local, pg, dev)
    # e2e through host buffers (pinned H2D of f, D2H of u and p inside the step)
    one_step(P.MIXED, e2e=True)          # untimed: first pinned-copy path
    e2e_times = [one_step(P.MIXED, e2e=True)[0] for _ in range(max(3, a.steps))]
    # FP64 V-cycle for the mixed-vs-FP64 comparison
    one_step(P.FP64)                     # untimed: FP64 warm-up
    f64 = [one_step(P.FP64) for _ in range(max(3, a.steps))]
    # the other relaxation, same step otherwise
    other = "v11" if a.relaxation == "v22" else "v22"
    one_step(P.MIXED, relax=other)
    alt = [one_step(P.MIXED, relax=other) for _ in range(max(3, a.steps))]
    paper = None
    if not a.no_paper_scale:
        try:
            paper = paper_scale_section(P, W, dev, stream, flush)
        except Exception as e:  # noqa: BLE001
            paper = {"error": str(e)[:300]}
    # FP64 pipe peak, measured live: a DFMA loop on every SM
    fp64_probe = {}
    try:
        P._binding.probe_fp64_peak(1 << 12, 2, stream=stream.cuda_stream)
        with Clocks(local) as pclk:
            runs = [P._binding.probe_fp64_peak(1 << 17, 2, stream=stream.cuda_stream) for _ in range(5)]
        tf = sorted(r[0] for r in runs)
        fp64_probe = {"median_tflops": tf[len(tf) // 2], "max_tflops": tf[-1], "min_tflops": tf[0],
                      "ms_per_launch": sorted(r[1] for r in runs)[len(runs) // 2], "launches": len(runs),
                      "clocks": pclk.summary()}
    except Exception as e:  # noqa: BLE001
        fp64_probe = {"error": str(e)[:200]}
    # solve-phase roofline: level 0's FP32 patch apply (one ASM sweep over
    # 4225 inverses), timed by CUDA events on its stream after an L2 flush
    hp = make(P.MIXED, 1 << P._binding.PROF_PATCH)
    n0 = hp.info()["n_free"][0]
    rr = torch.randn(n0, dtype=torch.float64, device=dev)
    k0 = hp.prof_read(P._binding.PROF_PATCH)[0]
    for _ in range(10):
        flush.fill_(1.0)
        hp.asm(0, rr, P.MIXED)
    torch.cuda.synchronize(dev)
    k1 = hp.prof_read(P._binding.PROF_PATCH)[0]
    patch_ms = sorted(hp.prof_read_one(P._binding.PROF_PATCH, i) for i in range(k0, k1))
    patch_ms = patch_ms[len(patch_ms) // 2] if patch_ms else 0.0     # median launch
    hp.close()
    batched = None
    if not a.no_batched:
        try:
            batched = batched_section(a, P, W, dev, stream, flush,
                                      json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
                                      if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0)
        except Exception as e:  # noqa: BLE001
            batched = {"error": str(e)[:300]}
        try:
            batched["buckets"] = buckets_section(a, P, W, dev, stream, flush)
        except Exception as e:  # noqa: BLE001
            batched["buckets"] = {"error": str(e)[:300]}
    fbf_res = None
    if not a.no_fbf:
        try:
            fbf_res = fbf_section(a, P, W, dev, stream, flush)
        except Exception as e:  # noqa: BLE001
            fbf_res = {"error": str(e)[:300]}
    highk = None
    if not a.no_highk:
        try:
            highk = highk_section(a, P, W, dev, stream, flush)
        except Exception as e:  # noqa: BLE001
            highk = {"error": str(e)[:300]}
    adj = None
    if not a.no_adjoint:
        try:
            adj = adjoint_section(a, P, W, dev, stream, flush)
        except Exception as e:  # noqa: BLE001
            adj = {"error": str(e)[:300]}
    barrier()
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    # dominant kernel of a step: the batched FP64 Gauss-Jordan patch inversion
    # (2 n_i^3 flop per patch; FP64 ALU bound on GB300)
    sizes = []
    flops_gj = 0.0
    # algorithmic flops of the factored saddle block inverse per patch (n_v
    # velocity nodes per component, n_p pressures, d components, z_c(q) the
    # nonzero rows of column q of B_c^T, z_c = sum_q z_c(q)):
    #   n_v^3 (sweep of L, upper triangle) + 2 n_v z_c per component
    #   (W_c = L^-1 B_c^T over B's nonzeros) + 2 sum_{q <= r} z_c(q) per
    #   component (S = B W, upper) + n_p^3 (sweep of S); the kernel skips the
    #   structural zeros of B (a pressure node couples only with the velocity
    #   nodes of its support cells); the stored form is (L^-1, W, S^-1), so
    #   X = W S^-1 and the explicit velocity block are not formed
    # algorithmic bytes of one FP32 saddle apply per patch: L^-1, W and S^-1
    # read once (leading dimensions rounded up to 4), the gathered residual,
    # the weights and the result (3 n_i floats)
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                       hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, host_only=1)
    flops_levels = []
    apply_bytes = []
    up4 = lambda x: (x + 3) // 4 * 4  # noqa: E731
    for li in range(stats["n_levels"] - 1):
        off, dofs = probe.patches(li)
        _, comp, _ = probe.level_dofs(li)
        K = probe.get_csr(li).tocsr()
        cd = comp[dofs]
        f = 0.0
        by = 0.0
        for pi in range(len(off) - 1):
            pd = dofs[off[pi]:off[pi + 1]]
            c = cd[off[pi]:off[pi + 1]]
            nv = float((c == 0).sum())
            npr = float((c == d).sum())
            f += nv ** 3 + npr ** 3
            pres = pd[c == d]
            for cc in range(d):
                zq = np.asarray((K[pd[c == cc]][:, pres] != 0).sum(axis=0)).ravel().astype(float)
                f += 2 * nv * zq.sum() + 2 * float((zq * (npr - np.arange(len(zq)))).sum())
            nvi, npi = int(nv), int(npr)
            # L^-1 as its packed upper triangle (the bulk-copy apply's layout)
            by += 4.0 * (up4(nvi * (nvi + 1) // 2) + up4(d * nvi) * npi + up4(npi) * npi) + 12.0 * (d * nvi + npi)
        flops_levels.append(f)
        apply_bytes.append(by)
        sizes.append(np.diff(off))
    flops_gj = sum(flops_levels)
    probe.close()
    gj_launches_per_step = gj_prof[0] / a.steps
    gj_ms_per_step = gj_prof[1] / a.steps
    # FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA lanes per
    # clock x 2 flop x 2.07 GHz = 1.259 TFLOP/s (the nominal 1.25 TFLOP/s);
    # the roofline uses the live DFMA-loop measurement (median of 5)
    fp64_derived_tflops = 152 * 2 * 2 * 2.07e9 / 1e12
    fp64_peak_tflops = fp64_probe["median_tflops"] if fp64_probe.get("median_tflops") else fp64_derived_tflops
    # dominant kernel: level 0's saddle block inversion launch (4225 patches)
    gj0_ms = sorted(gj0)[len(gj0) // 2] if gj0 else 0.0
    achieved_gj0 = flops_levels[0] / (gj0_ms * 1e-3) / 1e12 if gj0_ms > 0 else None
    achieved_gj = flops_gj / (gj_ms_per_step * 1e-3) / 1e12 if gj_ms_per_step > 0 else None
    # DRAM bytes of that launch from one ncu capture of the same kernel and
    # workload (dram__bytes_read.sum + dram__bytes_write.sum of the level-0
    # launch of the CSR-reading, sparse-B inversion)
    traffic_gj0 = (74.930176 + 31.753216) * 1e6 if a.workload == "th_p4_64x64" else None
    # level-0 FP32 saddle apply: algorithmic bytes (above)
    patch_bytes = apply_bytes[0]
    patch_gbs = patch_bytes / (patch_ms * 1e-3) / 1e9 if patch_ms > 0 else None
    line = {
        "metric": METRIC, "value": ms_max, "unit": "ms", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": step_config(a, w, world),
        "precision": "mixed (FP32 V-cycle, FP64 FGMRES/LU/coarse)",
        "problem": {"n_free": stats["n_free"], "nnz_level0": stats["nnz"][0],
                    "l2": "flushed (256 MB write) before every step", "inputs": "mesh on host, f resident in HBM"},
        "iterations": its_l[-1],
        "step_ms": {"min": min(times), "median": sorted(times)[len(times) // 2], "max": max(times)},
        "setup_ms": {k: round(stats[k], 3) for k in ("t_mesh_ms", "t_assembly_ms", "t_spaces_ms", "t_matrices_ms",
                                                     "t_patches_ms", "t_transfers_ms", "t_upload_ms", "t_launch_thread_ms", "t_launch_wait_ms", "t_upload_post_ms", "t_gather_lu_ms",
                                                     "t_coarse_ms", "t_eig_ms", "t_graph_ms", "t_total_ms")},
        "e2e": {"value": sum(e2e_times) / len(e2e_times), "unit": "ms",
                "h2d_bytes_per_step": int(f_host.numel() * 8),
                "d2h_bytes_per_step": int((u_host.numel() + p_host.numel()) * 8)},
        "fp64": {"value": sum(x[0] for x in f64) / len(f64), "unit": "ms", "iterations": f64[-1][1],
                 "setup_ms": f64[-1][3]["t_total_ms"]},
        "gpu_launches": int(launches / a.steps),
        "roofline": {"kernel": "saddle_inverse_smem, level-0 launch (4225 Vanka patches, FP64 factored saddle block "
                               "inverse)",
                     "bound": "alu", "achieved": achieved_gj0, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                     "frac": (achieved_gj0 / fp64_peak_tflops) if achieved_gj0 else None,
                     "traffic": traffic_gj0,
                     "peak_source": ("measured: DFMA loop (stokes_probe_fp64_peak, 8 FMA chains x 256 threads x 2 "
                                     "CTAs per SM), median of 5 launches in this run"
                                     if fp64_probe.get("median_tflops") else
                                     "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"),
                     "peak_derived": fp64_derived_tflops, "fp64_probe": fp64_probe,
                     "flop_per_launch": flops_levels[0], "ms_per_launch": gj0_ms,
                     "all_levels": {"launches_per_step": gj_launches_per_step, "ms_per_step": gj_ms_per_step,
                                    "flop_per_step": flops_gj, "achieved": achieved_gj}},
        "roofline_solve": {"kernel": "saddle_apply_bulk_f32, level 0 (one ASM sweep over the factored FP32 inverses, "
                                     "L^-1 packed, one bulk copy per patch)",
                           "bound": "hbm",
                           "achieved": patch_gbs, "peak": hbm, "unit": "GB/s",
                           "frac": (patch_gbs / hbm) if patch_gbs else None, "bytes_per_launch": patch_bytes,
                           "us_per_launch": 1e3 * patch_ms, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "wall_s_timed": wall,
    }
    line["speedup_mixed_vs_fp64"] = line["fp64"]["value"] / ms_max
    line["relaxation_" + other] = {"value": sorted(x[0] for x in alt)[len(alt) // 2], "unit": "ms",
                                   "iterations": alt[-1][1], "relaxation": relax_text(other)}
    if paper is not None:
        line["paper_scale"] = paper
    if batched is not None:
        line["batched"] = batched
    if adj is not None:
        line["adjoint"] = adj
    if fbf_res is not None:
        line["fbf"] = fbf_res
    if highk is not None:
        line["high_k"] = highk
    line["clocks"] = clk.summary()
    if not a.no_cpu_baseline and world == 1:
        try:
            npz = os.path.join(tempfile.gettempdir(), f"stokes_bench_oracle_{os.getpid()}.npz")
            o = run_oracle(a.workload, a.relaxation, save=npz)
            try:
                def solve_lib(prec, f_np, tol):
                    hh = make(prec)
                    uu, pp, _, _ = hh.solve(torch.tensor(f_np.reshape(-1), device=dev), tol=tol)
                    res = (uu.cpu().numpy(), pp.cpu().numpy())
                    hh.close()
                    return res
                line["oracle_error"] = oracle_error(P, W, w, npz, solve_lib)
            except Exception as e:  # noqa: BLE001
                line["oracle_error"] = {"error": str(e)[:200]}
            finally:
                if os.path.exists(npz):
                    os.remove(npz)
            host_cores = os.cpu_count() or 1
            line["cpu_baseline"] = {"value": 1e3 * (o["setup_s"] + o["solve_s"]), "unit": "ms", "cores": 1,
                                    "host_cores": host_cores, "kind": "oracle",
                                    "sample": f"one full setup + FGMRES solve of {a.workload} to {TOL}, "
                                              f"{relax_text(a.relaxation)}, single-threaded numpy/scipy",
                                    "iterations": o["its"],
                                    "setup_ms": 1e3 * o["setup_s"], "solve_ms": 1e3 * o["solve_s"]}
            try:
                oa = run_oracle(a.workload, a.relaxation, threads=host_cores)
                line["cpu_baseline"]["all_cores"] = {"value": 1e3 * (oa["setup_s"] + oa["solve_s"]), "unit": "ms",
                                                     "threads": host_cores, "iterations": oa["its"],
                                                     "note": "same oracle run with BLAS threads = host cores"}
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline"]["all_cores"] = {"error": str(e)[:200]}
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {e}"[:200]}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
