"""Benchmark: multigrid-preconditioned CG, DOF/s to relative residual 1e-8.

One step = one full solve of the 257^3-vertex workload (log10 k ~ U[-2,2] on
16^3 cell blocks, f ~ U[-1,1], 7 levels, V(2,2) with Chebyshev(2)-Jacobi,
dense Cholesky on the 3^3 coarsest level, float64 CG to ||r|| <= 1e-8 ||f||)
with inputs resident on the GPU.  The headline form runs the V-cycle in
float32 inside the float64 CG; the plain float64 form and the bfloat16-
coefficient form are timed the same way and reported beside it, each with its
relative error against the CPU float64 oracle's solution of the same problem.

The same line carries the 513^3 contrast-10^6 target solve with Galerkin
coarse operators (target_513_c1e6), the paper's solver configurations, the
end-to-end figure through the C ABI with host buffers, the per-iteration host
round trip, and the oracle timed on the host cores (a full solve, the second
of two identical ones).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) the ranks solve one problem together, decomposed into N
z-slabs (rank r holds slab r; halo planes, dot-product sums and the
agglomeration level travel over NCCL): strong scaling.  --replicas makes
every rank solve its own independent problem instead (seed + rank, weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mg_inputs as mi  # noqa: E402

METRIC = "MG-PCG DOF/s to rel. residual 1e-8 (mixed vs FP64) and smoother HBM GB/s vs peak"
WORKLOAD = "poisson257_c1e4"
HEADLINE = "mixed_fp32"
FORMS = ("mixed_fp32", "fp64", "mixed_bf16k")

# Algorithmic HBM bytes per interior point for one launch of each kernel class,
# as a function of the vector element size v and the three-coefficient bytes c
# (each array counted once per point: neighbour re-reads served from cache are
# not).  float32 smoothers recompute D^-1 from the six coefficients; the float64
# ones read it (dinv = v).  The finest level's post-smoothing is step 0 (reads
# x, b; writes x, d) and step 1 with rho = r.z fused (reads x, d, b, float64 r;
# writes z): cheb_step is their average.
def bytes_per_point(cls: str, v: int, c: int, degree: int = 2, fp64: bool = False, flexible: bool = False) -> float:
    dinv = v if fp64 else 0
    return {
        "cheb_zero": 3 * v + c + (v if degree > 2 else 0),  # read b, dinv, k; write x (and d)
        "cheb_step": 4 * v + c + dinv,                    # (x+b+k+x'+d) and (x+d+b+k+z), averaged
        "resid": 3 * v + c,                               # read x, b, k; write r
        "restrict": 9 * v,                                # per coarse point: read 8 fine r, write 1
        "prolong": 2 * v + v / 8,                         # read x, e/8; write x
        "cg_dir": 32 + v,                                 # read z, p, x; write p, x (float64 p, x)
        "cg_apply": 3 * 8 + 24,                           # read p, D, k64; write q (float64)
        "cg_upd": 24 + (0 if fp64 else 4) + (v if flexible else 0),  # read r, q (z); write r (, float32 b)
        "dot": 2 * v,                                     # read b, z
        "cast": 12,                                       # float64 r -> float32 b
    }[cls]


def form_sizes(form: str):
    return {"fp64": (8, 24), "mixed_fp32": (4, 12), "mixed_bf16k": (4, 6)}[form]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


# ---- replicas: every rank solves its own problem; only timing is combined
def replica_seed(spec, rank: int) -> int:
    """Seed of rank's independent problem (the workload's seed shifted by the rank)."""
    return spec["seed"] + rank


def max_over_ranks(x: float, device) -> float:
    """Largest value over all ranks (the timed region of the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_dofs_per_s(unknowns_per_rank: int, world: int, ms_per_step: float) -> float:
    """Unknowns solved by all ranks per second of the slowest rank's step."""
    return world * unknowns_per_rank / (ms_per_step * 1e-3)


L2_BYTES = 129e6


def l2_note(N: int) -> str:
    """How the timed steps avoid a warm L2: a float64 vector of N^3 points, the
    solve's working set about 20 of them."""
    vec = N ** 3 * 8
    if vec > L2_BYTES:
        return (f"no flush: inputs larger than L2 (each float64 vector {vec / 1e6:.0f} MB; "
                f"working set > {20 * vec / 1e9:.1f} GB)")
    return (f"warm L2: each float64 vector {vec / 1e6:.2f} MB, the whole working set stays in the "
            f"129 MB L2 (a small parity-size case, not a throughput claim)")


def config_dict(spec, n_ranks, name=None, face_rule=0, adjoint=False, coarse_op="rediscretised", slabs=1,
                decomposed=False, backend="nccl"):
    N = spec["N"]
    levels = 1
    M = N
    while (M - 1) % 2 == 0 and (M - 1) // 2 + 1 >= 5:
        M = (M - 1) // 2 + 1
        levels += 1
    d = {
        "workload": f"{name or WORKLOAD}: {N}^3 vertices ({(N - 2) ** 3} unknowns), log10 k ~ U[{spec['lo']:g},{spec['hi']:g}] "
                    f"on {spec['block']}^3 cell blocks, f ~ U[-1,1], {'arithmetic' if face_rule else 'harmonic'}-mean "
                    f"edge k, {levels} levels ({'Galerkin R A P' if coarse_op == 'galerkin' else 're-discretised'} coarse "
                    f"operators), V(2,2) Chebyshev(2)-Jacobi, 3^3 dense Cholesky, CG to rel. residual "
                    f"{spec['rtol']:g}" + ("; step = forward + adjoint solve with the cell gradient" if adjoint else ""),
        "l2": l2_note(N),
        "parallelism": (f"one problem over {n_ranks} GPUs, one z-slab per rank ({backend})" if decomposed
                        else ("replicas" if n_ranks > 1 else "single GPU")
                        + (f", solve decomposed into {slabs} z-slabs" if slabs > 1 else "")),
    }
    return d


# ------------------------------------------------------------------ oracle arms
def oracle_cores() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_sample(spec, iters_to_tol: int, sample_iters: int):
    """Time `sample_iters` oracle PCG iterations on the full workload; return
    (DOF/s to tolerance extrapolated by the iteration count, seconds, cores)."""
    import oracle
    dims = (spec["N"],) * 3
    k = mi.cell_k(dims, spec["block"], spec["lo"], spec["hi"], spec["seed"])
    f = mi.rhs_f(dims, spec["seed"])
    O = oracle.Oracle(k)
    t = time.perf_counter()
    O.pcg(f, 0.0, maxit=sample_iters)
    dt = time.perf_counter() - t
    n = (spec["N"] - 2) ** 3
    return n / (dt / sample_iters * iters_to_tol), dt, oracle_cores()


def oracle_full_solve(k, f, rtol):
    """The oracle's solve of the workload to tolerance, run twice with the
    second timed (the paper's protocol of timing the second of two identical
    solves).  Returns (solution, iterations, seconds of the second solve)."""
    import oracle
    O = oracle.Oracle(k)
    O.pcg(f, rtol, maxit=3000)
    t = time.perf_counter()
    x, it, _ = O.pcg(f, rtol, maxit=3000)
    return x, it, time.perf_counter() - t


def golden_iterations():
    with open(os.path.join(ROOT, "tests", "golden", "oracle_solves.json")) as fh:
        return json.load(fh)[WORKLOAD]["iterations"]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    spec = dict(mi.WORKLOADS[WORKLOAD])
    its = golden_iterations()
    sample = 4
    vals, times = [], []
    for s in range(args.warmup + args.steps):
        v, dt, cores = oracle_sample(spec, its, sample)
        if s >= args.warmup:
            vals.append(v)
            times.append(dt)
    value = float(np.median(vals))
    desc = (f"CPU FP64 oracle (assembled CSR, OpenMP) on the full {spec['N']}^3 workload: each step times "
            f"{sample} PCG iterations and the value is EXTRAPOLATED to a solve by its recorded {its}-iteration count "
            f"to tolerance (a full solve per step would take about 20 s on 16 cores; the full-solve figure is the "
            f"GPU arm's cpu_baseline)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.median(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "precision": "fp64 (CPU oracle)", "iterations": its,
        "config": config_dict(spec, 1),
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import paper_1604_07163_gb300 as mg

    rank, world, local = dist_env()
    # ranks beyond the visible devices share them (only for checking the
    # multi-rank path on fewer GPUs, with MG_BENCH_BACKEND=gloo: NCCL needs one
    # device per rank)
    dev = torch.device("cuda", local % max(torch.cuda.device_count(), 1) if world > 1 else 0)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(os.environ.get("MG_BENCH_BACKEND", "nccl"))
    spec = dict(mi.WORKLOADS[args.workload])
    decomposed = world > 1 and not args.replicas  # one problem over all ranks, one z-slab each
    seed = spec["seed"] if decomposed else replica_seed(spec, rank)
    dims = (spec["N"],) * 3
    n = (spec["N"] - 2) ** 3
    k_np = mi.cell_k(dims, spec["block"], spec["lo"], spec["hi"], seed)
    f_np = mi.rhs_f(dims, seed)
    k = torch.tensor(k_np, device=dev)
    f_host = torch.tensor(f_np).pin_memory()
    f = f_host.to(dev)
    rtol = spec["rtol"]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    step_medians = {}

    def timed(fn, steps, key=None):
        """Device time of `steps` calls of fn (CUDA events on the current
        stream, barrier and synchronize on both sides), max over ranks, ms
        per call.  An event between consecutive calls also gives each call's
        own time; with key, their median (max over ranks) is kept in
        step_medians[key]."""
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record()
        out = []
        for i in range(steps):
            out.append(fn())
            ev[i + 1].record()
        barrier()
        if key is not None:
            per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
            step_medians[key] = max_over_ranks(per[len(per) // 2], dev)
        return max_over_ranks(ev[0].elapsed_time(ev[steps]), dev) / steps, out

    forms = {}
    solutions = {}
    roofline = smoother = clocks = host_gap = e2e = None
    launches = 0
    run_forms = [HEADLINE] + [fm for fm in args.forms.split(",") if fm in FORMS and fm != HEADLINE]

    def new_solver(kk, **kw):
        """A solver of the run's parallel layout: in the decomposed run this
        rank's slab of the z-slab decomposition, connected to the others."""
        if decomposed:
            kw.update(slabs=world, slab_rank=rank)
        S = mg.MGSolver(kk, mg.Params(**kw))
        if decomposed:
            S.attach_transport()
        return S

    phi_obs = None
    if args.adjoint:  # loss 0.5 |phi - phi_obs|^2 with phi_obs from the k field of seed + 1
        kobs = torch.tensor(mi.cell_k(dims, spec["block"], spec["lo"], spec["hi"], seed + 1), device=dev)
        So = new_solver(kobs, precision=HEADLINE, face_rule=args.face_rule, maxit=args.maxit,
                        coarse_op=args.coarse_op)
        phi_obs, _ = So.solve(f, rtol, raise_on_error=False)
        So.close()
        del So

    def dofs_per_s(ms):
        return n / (ms * 1e-3) if decomposed else whole_job_dofs_per_s(n, world, ms)

    def step(S):
        x, st = S.solve(f, rtol, raise_on_error=False)
        if args.adjoint:
            S.solve_adjoint((x - phi_obs).contiguous(), rtol, x)
        return x, st

    for form in (run_forms if not (args.only_paper_configs or args.only) else []):
        S = new_solver(k, precision=form, maxit=args.maxit, face_rule=args.face_rule, coarse_op=args.coarse_op,
                       **({} if decomposed else dict(slabs=args.slabs)))
        headline = form == HEADLINE
        # per-kernel timing instruments the single-domain solve; the
        # decomposed run's kernels are the same and are measured on one GPU
        instrument = headline and not decomposed
        profile_all = None
        for w in range(args.warmup):
            if instrument and w == 0:
                S.timing(True)  # one fully instrumented warm-up solve: per-kernel breakdown
            step(S)
            if instrument and w == 0:
                profile_all = S.kernel_times()
                S.timing(False)
        if headline:
            if instrument:
                dom = max(((c, v[0]) for (c, l), v in profile_all.items() if l == 0 and c != "host_gap"),
                          key=lambda t: t[1])[0]
            sampler = ClockSampler(dev.index if dev.index is not None else 0)
            sampler.start()
        ms, outs = timed(lambda: step(S), args.steps, key=form)
        x, st = outs[-1]
        forms[form] = {"value": dofs_per_s(ms), "ms_per_step": ms, "ms_per_step_median": step_medians[form],
                       "iters": st.iters, "true_rel_resid": st.true_rel_resid, "status": st.status}
        solutions[form] = x.detach().clone()
        if headline:
            launches = sum(o[1].kernel_launches for o in outs)
        if instrument:
            # the same K steps again with CUDA events around every launch of the
            # dominant finest-level kernel class and of the smoother steps (events
            # inside the V-cycle graph slow the whole solve, so the headline steps
            # above run without them)
            S.timing(True, classes=[dom] if dom == "cheb_step" else [dom, "cheb_step"], levels=[0])
            for _ in range(args.steps):
                S.solve(f, rtol, raise_on_error=False)
            torch.cuda.synchronize()
            kt = S.kernel_times()
            # and once more timing only the host round trip between outer
            # iterations (the V-cycle still replays from its graph)
            S.timing(True, classes=["host_gap"], levels=[0])
            ms_gap_run, gouts = timed(lambda: S.solve(f, rtol, raise_on_error=False), args.steps)
            gt = S.kernel_times().get(("host_gap", 0))
            S.timing(False)
        if headline:
            clocks = sampler.stop()
        if instrument:
            roofline = roofline_from(kt, form, clocks, dom, args.workload)
            smoother = roofline_from(kt, form, clocks, "cheb_step", args.workload)
            if roofline and roofline["bound"] == "alu":
                # the rate of a float64 FMA-chain kernel on this GPU now, beside
                # the peak derived from unit counts and the sampled clock: a
                # lower bound on what the float64 pipe sustains, not its peak
                fm = fp64_fma_peak()
                if fm:
                    roofline["fp64_probe_tflops"] = fm
                    roofline["frac_of_probe"] = roofline["achieved"] / fm
                    roofline["fp64_probe_source"] = (
                        "mg_fp64_fma_peak: independent float64 FMA chains on every SM, fastest of 5 launches "
                        "of about 16 ms, in this run after the timed steps; a lower bound on the float64 "
                        "pipe's rate (the operator itself exceeds it on long launches), not a peak")
            if gt:
                gap_ms, gap_n, _ = gt
                host_gap = {"us_per_iteration": 1e3 * gap_ms / gap_n, "ms_per_solve": gap_ms / args.steps,
                            "share_of_solve": (gap_ms / args.steps) / ms_gap_run, "iterations_measured": gap_n,
                            "what": "device time from the end of an outer iteration's last kernel to the next "
                                    "V-cycle launch (read of the CG scalars, host convergence test, next launch), "
                                    "V-cycle replayed from its CUDA graph"}
            forms[form]["kernel_ms_per_solve_warmup_profile"] = {f"{c}@L{l}": round(v[0], 4)
                                                                  for (c, l), v in profile_all.items()}
        if headline:
            # end to end through the C ABI with HOST buffers: the library copies the
            # pinned f in and x out inside every call
            x_host = torch.empty(dims, dtype=torch.float64).pin_memory()
            S.solve_host(f_host, x_host, rtol, raise_on_error=False)  # first call allocates the staging arrays
            if args.adjoint:
                def e2e_step():
                    S.solve_host(f_host, x_host, rtol, raise_on_error=False)
                    xe = x_host.to(dev, non_blocking=True)
                    S.solve_adjoint((xe - phi_obs).contiguous(), rtol, xe)
            else:
                def e2e_step():
                    S.solve_host(f_host, x_host, rtol, raise_on_error=False)
            ms_e2e, _ = timed(e2e_step, args.steps)
            e2e = {"value": dofs_per_s(ms_e2e), "unit": "DOF/s",
                   "h2d_bytes_per_step": f_host.numel() * 8, "d2h_bytes_per_step": x_host.numel() * 8,
                   "api": "mg_solve_host (C ABI, pinned host f and x)"}
        S.close()
        del S

    def timed_variant(**extra):
        """The headline precision with other method choices, on the same problem
        and tolerance, timed like the forms above."""
        S = mg.MGSolver(k, mg.Params(precision=HEADLINE, maxit=args.maxit, face_rule=args.face_rule, **extra))
        for _ in range(args.warmup):
            S.solve(f, rtol, raise_on_error=False)
        msg, outs = timed(lambda: S.solve(f, rtol, raise_on_error=False), args.steps)
        xg, stg = outs[-1]
        out = {"value": whole_job_dofs_per_s(n, world, msg), "unit": "DOF/s", "ms_per_step": msg,
               "iters": stg.iters, "true_rel_resid": stg.true_rel_resid, "status": stg.status,
               "precision": HEADLINE, **{k_: v_ for k_, v_ in extra.items() if k_ != "maxit"}}
        ref = solutions.get(HEADLINE)
        if ref is not None:
            out["rel_err_vs_headline_solution"] = float((xg - ref).norm() / ref.norm())
        S.close()
        del S
        return out

    if args.only:
        out_v = timed_variant(**VARIANTS[args.only])
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": "DOF/s", "variant": args.only, "result": out_v,
                              "config": config_dict(spec, world, args.workload)}), flush=True)
        return

    slabs = None
    if world == 1 and not args.adjoint and not args.no_slabs and args.slabs == 1 and not args.only_paper_configs:
        # the z-slab decomposition of the headline solve on this one GPU (slabs
        # run one after another, each halo exchange a device copy): its cost
        # over the single-domain solve and its distance from that solution
        slabs = {}
        for nsl in (2, 4):
            out_s = timed_variant(slabs=nsl, coarse_op=args.coarse_op)
            slabs[f"slabs{nsl}"] = out_s
    galerkin = paper = None
    if args.coarse_op == "rediscretised" and not args.adjoint and not args.no_galerkin and not decomposed:
        galerkin = timed_variant(**VARIANTS["galerkin"])
    if args.coarse_op == "rediscretised" and not args.adjoint and not args.no_paper_configs and not decomposed:
        # the solver configurations of the paper's experiments (Sec. 5): FGMRES
        # preconditioned by one V-cycle; Galerkin coarse operators with
        # Richardson(8)-Jacobi smoothing and the inexact coarsest GMRES-Jacobi
        # solve to 1e-4 (the truncation runs); re-discretised coarse operators
        # with Chebyshev(10)-Jacobi smoothing (the comparison runs, here with the
        # exact coarsest solve in place of their block-Jacobi/ILU(0) one)
        paper = {name: timed_variant(**VARIANTS[name])
                 for name in ("fgmres_galerkin_richardson8_gmres_coarse", "fgmres_rediscretised_chebyshev10")}
    if args.only_paper_configs:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": "DOF/s", "galerkin_coarse_operators": galerkin,
                              "paper_configurations": paper, "config": config_dict(spec, world, args.workload)}),
                  flush=True)
        return

    speedup = None
    if "fp64" in solutions:
        ref = solutions["fp64"]
        for form in run_forms:
            if form != "fp64":
                forms[form]["rel_err_vs_fp64_gpu"] = float((solutions[form] - ref).norm() / ref.norm())
        speedup = forms["fp64"]["ms_per_step"] / forms[HEADLINE]["ms_per_step"]

    target = None
    if (world == 1 and not args.no_target_513 and args.workload == WORKLOAD and not args.adjoint
            and args.coarse_op == "rediscretised"):
        target = target_513_c1e6(args, dev, timed)

    cpu = None
    if (rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD and not args.adjoint
            and args.coarse_op == "rediscretised"):
        xo, ito, dt = oracle_full_solve(k_np, f_np, rtol)
        cpu = {"value": n / dt, "unit": "DOF/s", "cores": oracle_cores(), "kind": "oracle",
               "iterations": ito, "seconds": dt,
               "sample": f"full solve of the {spec['N']}^3 workload to rel. residual {rtol:g} by the CPU FP64 "
                         f"oracle ({ito} PCG iterations, {dt:.1f} s), the second of two identical solves"}
        xo_norm = np.linalg.norm(xo)
        for form, xs in solutions.items():
            forms[form]["rel_err_vs_oracle"] = float(np.linalg.norm(xs.cpu().numpy() - xo) / xo_norm)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": forms[HEADLINE]["value"], "unit": "DOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms[HEADLINE]["ms_per_step"],
        "higher_is_better": True, "scaling": "strong" if decomposed else "weak", "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic", "precision": HEADLINE, "iterations": forms[HEADLINE]["iters"],
        "config": config_dict(spec, world, args.workload, args.face_rule, args.adjoint, args.coarse_op,
                              world if decomposed else args.slabs, decomposed,
                              dist.get_backend() if world > 1 else "nccl"),
        "forms": forms, "speedup_mixed_vs_fp64": speedup, "target_513_c1e6": target,
        "galerkin_coarse_operators": galerkin, "paper_configurations": paper, "slab_decomposition": slabs,
        "roofline": roofline, "smoother_roofline": smoother, "host_gap": host_gap, "cpu_baseline": cpu,
        "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def target_513_c1e6(args, dev, timed):
    """The 513^3 contrast-10^6 target with Galerkin coarse operators: the
    float32-V-cycle and float64 forms, one warm-up and two timed solves each,
    their iterations and true residuals (also from the oracle's own operator),
    the speed-up of the mixed form at equal final accuracy, and the smoother
    step's HBM roofline at this size."""
    import torch
    import oracle
    import paper_1604_07163_gb300 as mg
    name = "poisson513_c1e6"
    spec = dict(mi.WORKLOADS[name])
    dims = (spec["N"],) * 3
    n = (spec["N"] - 2) ** 3
    k_np = mi.cell_k(dims, spec["block"], spec["lo"], spec["hi"], spec["seed"])
    f_np = mi.rhs_f(dims, spec["seed"])
    k = torch.tensor(k_np, device=dev)
    f = torch.tensor(f_np, device=dev)
    out = {"workload": config_dict(spec, 1, name, coarse_op="galerkin")["workload"], "steps": 2, "warmup": 1,
           "forms": {}}
    xs = {}
    for form in ("mixed_fp32", "fp64"):
        S = mg.MGSolver(k, mg.Params(precision=form, coarse_op="galerkin", maxit=args.maxit))
        S.solve(f, spec["rtol"], raise_on_error=False)
        ms, outs = timed(lambda: S.solve(f, spec["rtol"], raise_on_error=False), 2)
        x, st = outs[-1]
        out["forms"][form] = {"value": n / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms, "iters": st.iters,
                              "true_rel_resid": st.true_rel_resid, "status": st.status,
                              "setup_s": st.setup_s}
        if form == "mixed_fp32":
            S.timing(True, classes=["cheb_step"], levels=[0])
            S.solve(f, spec["rtol"], raise_on_error=False)
            torch.cuda.synchronize()
            out["smoother_roofline"] = roofline_from(S.kernel_times(), form, None, "cheb_step", name)
            S.timing(False)
        xs[form] = x.cpu().numpy()
        del x, outs
        S.close()
        del S
        torch.cuda.empty_cache()
    del k, f
    torch.cuda.empty_cache()
    O = oracle.Oracle(k_np)  # the finest operator is the same under either coarse-operator choice
    fn = np.linalg.norm(f_np)
    for form, xv in xs.items():
        r = (f_np - O.apply(xv))[1:-1, 1:-1, 1:-1]
        out["forms"][form]["true_rel_resid_by_oracle"] = float(np.linalg.norm(r) / fn)
    out["rel_err_mixed_vs_fp64_gpu"] = float(np.linalg.norm(xs["mixed_fp32"] - xs["fp64"]) / np.linalg.norm(xs["fp64"]))
    out["speedup_mixed_vs_fp64"] = out["forms"]["fp64"]["ms_per_step"] / out["forms"]["mixed_fp32"]["ms_per_step"]
    return out


# float64 operations per point of the float64-pipe-bound outer-CG kernel
# (6 FMA for the neighbour sum, 1 for D p - S, 1 for p.q)
# Method variants timed beside the headline solve (same problem, precision and
# tolerance): Galerkin coarse operators, and the two solver configurations of
# the paper's Sec. 5 experiments.
VARIANTS = {
    "galerkin": dict(coarse_op="galerkin"),
    "fgmres_galerkin_richardson8_gmres_coarse": dict(krylov="fgmres", coarse_op="galerkin", smoother="richardson",
                                                     nu_pre=8, nu_post=8, coarse_solve="gmres", coarse_rtol=1e-4),
    "fgmres_rediscretised_chebyshev10": dict(krylov="fgmres", cheby_degree=10),
}
CG_APPLY_FLOPS = 16
# GB300: 152 SMs x 2 float64 FMA per clock per SM (the nominal 1.25 TFLOP/s at 2.07 GHz)
FP64_FLOP_PER_SM_CLK = 4

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# finest-level kernel classes, from one ncu capture each on the 257^3 workload
# (profiles/ holds the summaries), keyed by the hash of the CUDA sources they
# were captured with: once the sources change the figure no longer describes
# the kernel and traffic is reported as null.
NCU_TRAFFIC = {
    # (workload, form, class): (DRAM bytes per launch, CUDA-source hash at capture)
    # cheb_step: mean of the two finest-level launches per V-cycle (step 0:
    # 450.1 MB; step 1 with b.z: 460.8 MB)
    ("poisson257_c1e4", "mixed_fp32", "cheb_step"): (455.5e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "cheb_zero"): (396.5e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "resid"): (392.4e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "prolong"): (79.0e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "restrict"): (66.9e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "cg_apply"): (788.8e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "cg_dir"): (547.4e6, "f8447c71119a0be7"),
    ("poisson257_c1e4", "mixed_fp32", "cg_upd"): (413.4e6, "f8447c71119a0be7"),
}


def code_tokens(text: str) -> str:
    """CUDA/C++ source with comments removed and whitespace collapsed: what
    the compiler sees (string literals in these sources hold no comment
    markers), so that editing a comment does not change the hash below."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


# Sources that hold none of the measured kernels: the float64 FMA-rate probe
# (mg_peak.cu) is compiled on its own and shares no code with the solver, so
# it does not invalidate the traffic figures.
HASH_EXCLUDED = ("mg_peak.cu",)


def csrc_hash(sources=None) -> str:
    """Hash of the CUDA sources' code (comments and layout excluded).
    sources: {file name: text}; default the files of the package's csrc/."""
    import hashlib
    if sources is None:
        d = os.path.join(ROOT, "paper_1604_07163_gb300", "csrc")
        sources = {}
        for fn in os.listdir(d):
            if fn.endswith((".cu", ".cuh")) and fn not in HASH_EXCLUDED:
                with open(os.path.join(d, fn), encoding="utf-8") as fh:
                    sources[fn] = fh.read()
    h = hashlib.sha256()
    for fn in sorted(sources):
        h.update(fn.encode())
        h.update(code_tokens(sources[fn]).encode())
    return h.hexdigest()[:16]


def measured_traffic(workload, form, cls):
    rec = NCU_TRAFFIC.get((workload, form, cls))
    if rec is None or rec[1] != csrc_hash():
        return None
    return rec[0]


def fp64_fma_peak(launches=5):
    """Rate of the library's float64 FMA-chain probe on the current GPU in
    TFLOP/s (a lower bound on the float64 pipe's rate), or None."""
    import ctypes
    from paper_1604_07163_gb300 import _lib
    r = ctypes.c_double()
    rc = _lib.load().mg_fp64_fma_peak(launches, ctypes.byref(r))
    return r.value if rc == 0 else None


def roofline_from(kt, form, clocks, cls, workload):
    """Roofline entry of level-0 kernel class cls from the live CUDA-event
    timing: algorithmic GB/s vs the measured HBM peak, or float64 FLOP/s vs
    the float64 pipe peak for the float64-pipe-bound outer-CG operator."""
    rec = kt.get((cls, 0))
    if rec is None:
        return None
    ms, nl, pts = rec
    avg_s = ms * 1e-3 / nl
    traffic = measured_traffic(workload, form, cls)
    if cls == "cg_apply":
        mhz = clocks["sm_mhz"] if clocks else 2070.0
        fpeak = 152 * FP64_FLOP_PER_SM_CLK * mhz * 1e6 / 1e12
        flops = CG_APPLY_FLOPS * pts / nl
        ach = flops / avg_s / 1e12
        return {"bound": "alu", "kernel": cls, "achieved": ach, "peak": fpeak, "unit": "TFLOP/s",
                "frac": ach / fpeak, "peak_source": "derived: 152 SMs x 4 float64 flop/clk x median SM clock",
                "traffic": traffic, "algorithmic_flops_per_launch": flops, "avg_launch_ms": ms / nl, "launches": nl}
    v, c = form_sizes(form)
    peak, which = load_peaks()
    bpp = bytes_per_point(cls, v, c, fp64=form == "fp64")
    alg = bpp * pts / nl  # restrict: pts are coarse points
    achieved = alg / avg_s / 1e9
    return {"bound": "hbm", "kernel": cls, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": which, "traffic": traffic,
            "algorithmic_bytes_per_launch": alg, "avg_launch_ms": ms / nl, "launches": nl}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default=",".join(FORMS),
                    help="comma-separated subset of " + ",".join(FORMS) + " (the headline form is always run)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(mi.WORKLOADS),
                    help="synthetic workload (the headline metric is quoted on " + WORKLOAD + ")")
    ap.add_argument("--face-rule", type=int, default=0, help="edge k: 0 harmonic (default), 1 arithmetic mean")
    ap.add_argument("--coarse-op", default="rediscretised", choices=["rediscretised", "galerkin"],
                    help="coarse operators: re-discretised (default) or Galerkin R A P")
    ap.add_argument("--no-galerkin", action="store_true",
                    help="skip the extra timing of the headline form with Galerkin coarse operators")
    ap.add_argument("--no-paper-configs", action="store_true",
                    help="skip timing the solver configurations of the paper's experiments")
    ap.add_argument("--no-target-513", action="store_true",
                    help="skip the 513^3 contrast-10^6 Galerkin target solve")
    ap.add_argument("--only-paper-configs", action="store_true",
                    help="time only the Galerkin variant and the paper's solver configurations (for profiling)")
    ap.add_argument("--only", choices=sorted(VARIANTS),
                    help="time only this one method variant of the headline precision (for profiling)")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: every rank solves its own problem instead of one decomposed problem")
    ap.add_argument("--slabs", type=int, default=1,
                    help="solve every form with the z-slab decomposition into this many slabs (1: none)")
    ap.add_argument("--no-slabs", action="store_true",
                    help="skip timing the headline form decomposed into 2 and 4 z-slabs")
    ap.add_argument("--maxit", type=int, default=3000)
    ap.add_argument("--adjoint", action="store_true", help="each step is a forward + adjoint solve with gradient")
    args = ap.parse_args()
    if args.warmup < 3 and args.workload == WORKLOAD:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
