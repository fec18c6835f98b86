"""Benchmark: homogenised designs/sec (6x6 C^H) on synthetic shell designs.

One step = the whole path for one design: field -> distance -> threshold ->
mask -> six periodic cell problems (FP32 PCG with a multigrid preconditioner
+ FP64 residual refinement to a relative residual of --tol, default 1e-7) ->
C^H, through the C-ABI call shl_homogenize.  The metric asks C^H within 1e-4
(relative entry error); every timed design is solved again afterwards,
untimed, by the FP64 GPU path (FP64 CG and residuals) to 1e-11 and the
largest entry error is reported ("accuracy").

Default workload: 64^3 grid, 32 charges uniform in the cell with magnitudes
N(0,1), 8 % solid volume (seeded synthetic designs; the paper's datasets are
not available).  Multi-GPU: independent replicas (designs are independent),
one process per GPU, weak scaling, no data-path collective.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl shl|reference]
  python bench.py --serve [--requests R] [--slots S]   # serving stream
  python bench.py --kernel apply [--r R]              # dominant kernel alone
  python bench.py --field                              # field on the paper's Table 1 shapes
  python bench.py --grad [--batch B]                   # inverse-design gradients at 64^3
  python bench.py --design [--objective Keff] [--steps K]  # inverse-design driver at 64^3
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, r, description)
    "gaussian64": ("gaussian_64", 64, "64^3 grid, 32 charges uniform, q~N(0,1), 8% solid"),
    "cubic128": ("cubic_128", 128, "128^3 grid, 48 charges (O_h orbit), 5% solid"),
    "plain32": ("plain_32", 32, "32^3 grid, 8 charges +-1, 15% solid"),
    "shell256": ("shell_256", 256, "256^3 grid, 32 charges +-1, half-thickness t = 0.02 (timing-table setting)"),
}
APPLY_BYTES_PER_NODE_F32 = 72 + 72 + 1  # read p (18 floats), write q (18 floats), 1 mask byte
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) per launch of the FP32 stiffness apply at 64^3
# (the row kernel), from one `ncu --set full` capture of
# `bench.py --kernel apply --r 64`: reads 19,177,472 B (p and the mask, the
# algorithmic minimum) + 0 B written (q's writes were still in L2 when the
# captured launch ended).  Reset to None whenever the kernel changes.
APPLY_TRAFFIC_64 = 19_177_472


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(design, r, golden_iters):
    """The FP64 oracle as it stands on a bounded sample of one design: full
    field/voxelisation, assembly, a fixed number of PCG iterations and C^H,
    scaled to a whole design by the oracle's own iteration count."""
    import oracle
    t0 = time.perf_counter()
    vox = oracle.voxelize(design, r)
    t_vox = time.perf_counter() - t0
    rho = vox["mask"].astype(np.float64)
    t0 = time.perf_counter()
    oracle.solve(r, rho, tol=1e-300, maxit=0)
    t_setup = time.perf_counter() - t0
    n_s = 60
    t0 = time.perf_counter()
    u, *_ = oracle.solve(r, rho, tol=1e-300, maxit=n_s)
    t_it = (time.perf_counter() - t0 - t_setup) / n_s
    t0 = time.perf_counter()
    oracle.chom(r, rho, u)
    t_c = time.perf_counter() - t0
    per_design = t_vox + t_setup + golden_iters * t_it + t_c
    sample = (f"oracle on one {r}^3 design: field+voxelise, assembly, {n_s} PCG iterations and C^H timed; "
              f"iterations scaled to {golden_iters} (the oracle's own count to 1e-12 on the seed-0 design)")
    return 1.0 / per_design, per_design, sample, oracle.num_threads()


def oracle_validate():
    """One fully converged oracle solve (32^3, 8 charges, 15 % solid, to
    1e-12), timed whole, beside the sample model's prediction for the same
    design (the model times 60 iterations and scales by the iteration count):
    the ratio measured / predicted checks the scaling the baseline rests on."""
    import oracle
    from paper_2511_04025_b300 import inputs
    d, r = inputs.plain_32(0), 32
    t0 = time.perf_counter()
    res = oracle.homogenize(d, r, tol=1e-12)
    full = time.perf_counter() - t0
    _, predicted, _, cores = oracle_sample(d, r, int(max(res["iters"])))
    return {"design": "plain_32 seed 0 (32^3)", "iters": int(max(res["iters"])), "measured_s": full,
            "predicted_s": predicted, "ratio": full / predicted, "cores": cores}


def golden_iters(workload):
    fn = os.path.join(ROOT, "tests", "golden", {"gaussian64": "gaussian64_s0", "plain32": "plain32_s0"}
                      .get(workload, "gaussian64_s0") + ".json")
    try:
        with open(fn) as f:
            return int(max(json.load(f)["iters"]))
    except Exception:
        return 5000


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    return rank, world, local


def max_over_ranks(world, *vals):
    """Each value's largest over the ranks (the job takes as long as its
    slowest replica; errors are as large as the worst one)."""
    if world <= 1:
        return tuple(float(v) for v in vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return tuple(float(v) for v in t)


def rank_seeds(rank, n):
    """Design seeds of one replica: disjoint across ranks (rank r uses
    100000 r + i), so the job's designs are all different."""
    return [100000 * rank + i for i in range(n)]


def job_rate(world, steps, per_step, seconds):
    """Whole-job throughput: every rank did steps x per_step designs in the
    (max-over-ranks) time."""
    return world * steps * per_step / seconds


def bench_config(args, r, desc, world):
    """The workload the headline line is quoted on (both arms print it)."""
    B = max(1, args.batch_designs)
    return {"workload": args.workload, "desc": desc + (", active set (void culled)" if args.active else ""), "r": r,
            "precision": args.precision, "tol": args.tol,
            "l2": "flushed between steps", "parallelism": f"replicas x{world}",
            "batch": f"{B} designs per step, concurrent on {min(B, args.slots)} serving slots"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, each step a bounded sample."""
    rank, world, local = dist_setup(args.gpus)
    if rank != 0:
        return
    from paper_2511_04025_b300 import inputs
    gen, r, desc = WORKLOADS[args.workload]
    gi = golden_iters(args.workload)
    for i in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps are not needed
    times, walls = [], []
    sample = cores = None
    for i in range(args.steps):
        d = getattr(inputs, gen)(i)
        t0 = time.perf_counter()
        v, per, sample, cores = oracle_sample(d, r, gi)
        walls.append(time.perf_counter() - t0)
        times.append(per)
    value = args.steps / sum(times)
    # ms_per_step is the measured time of one step (one bounded sample); the
    # designs/s value extrapolates each sample to a whole design
    line = {"metric": "homogenized designs/sec", "value": value, "unit": "designs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "s_per_design_extrapolated": float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": bench_config(args, r, desc, world),
            "cpu_baseline": {"value": value, "unit": "designs/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "extrapolated": True},
            "e2e": {"value": value, "unit": "designs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_apply(h, r, design, stream, launches=40):
    """Average duration of one FP32 stiffness apply (6 load cases) on the
    design's mask, CUDA events on the launch stream.  The launches rotate over
    enough (p, q) pairs that the working set exceeds the 126 MB L2, so every
    launch streams its operands from HBM."""
    import torch
    from paper_2511_04025_b300 import shl
    N = r ** 3
    mask = torch.empty(N, dtype=torch.uint8, device="cuda")
    shl.shl_voxelize(h, design, r, mask=mask, stream=stream)
    per_set = 2 * 18 * N * 4
    nsets = max(1, -(-(320 << 20) // per_set))
    ps = [torch.randn(18, N, dtype=torch.float32, device="cuda") for _ in range(nsets)]
    qs = [torch.empty_like(p) for p in ps]
    torch.cuda.synchronize()
    for i in range(3 * nsets):
        shl.shl_apply(h, r, ps[i % nsets], qs[i % nsets], mask=mask, stream=stream)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # hold the stream while the host enqueues every launch, so that the events
    # time the kernels back to back and not the host's launch rate
    with torch.cuda.stream(stream):
        torch.cuda._sleep(40_000_000)
    a0.record(stream)
    for i in range(launches):
        shl.shl_apply(h, r, ps[i % nsets], qs[i % nsets], mask=mask, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / 1e3 / launches


ROW_GRIDS = (32, 48, 64, 96, 128, 256)  # grids the FP32 row kernel serves (others: the tile kernel)


def apply_roofline(r, apply_s):
    peak, peak_kind = peaks()
    achieved = APPLY_BYTES_PER_NODE_F32 * r ** 3 / apply_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": APPLY_TRAFFIC_64 if r == 64 else None, "kernel": (f"apply_rows_kernel<{r}> (FP32 stiffness apply)" if r in ROW_GRIDS
                       else "apply_kernel<float> (FP32 stiffness apply)"),
            "peak_kind": peak_kind, "launch_us": apply_s * 1e6, "operands": "HBM (rotating > L2)"}


def run_kernel(args):
    """The dominant kernel alone: FP32 stiffness apply on the workload's first
    design at grid size --r (default: the workload's)."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    torch.cuda.set_device(0)
    gen, r0, _ = WORKLOADS[args.workload]
    r = args.r or r0
    with shl.Context(0) as ctx:
        stream = torch.cuda.Stream()
        apply_s = time_apply(ctx.handle, r, getattr(inputs, gen)(0), stream, launches=args.launches)
    line = {"kernel": "apply", "r": r, "workload": args.workload, "launches": args.launches,
            "roofline": apply_roofline(r, apply_s)}
    print(json.dumps(line), flush=True)


# Table 1 of the paper: field evaluation shapes (r, 2N) and the H200 times it
# reports (context only; another machine, another method).
FIELD_SHAPES = [(64, 32), (128, 32), (256, 32), (256, 64), (256, 128), (256, 256)]
FIELD_PAPER_H200_MS = {(64, 32): 0.7, (128, 32): 5.5, (256, 32): 43.0, (256, 64): 85.8, (256, 128): 171.7,
                       (256, 256): 347.2}
FP64_NOMINAL_GFLOPS = 1250.0  # B300 FP64 (non-tensor), nominal


def run_field(args):
    """Field throughput on the paper's Table 1 shapes: F and grad F of 2N
    balanced charges on the r^3 voxel centres (K = 3), FP64, CUDA events on
    the launch stream.  The separable evaluation costs 4(2K+1) FMAs per voxel
    after per-plane and per-line contractions, independent of 2N."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    torch.cuda.set_device(0)
    rows = []
    with shl.Context(0) as ctx:
        h = ctx.handle
        fp64_peak = shl.shl_probe_peaks(h)["fp64_fma_gflops"]
        stream = torch.cuda.Stream()
        for r, n in FIELD_SHAPES:
            d = inputs.random_design(7, n, 0.1)
            F = torch.empty(r ** 3, dtype=torch.float64, device="cuda")
            gF = torch.empty(r ** 3, 3, dtype=torch.float64, device="cuda")
            for _ in range(3):
                shl.shl_field(h, d, r, F, gF, stream=stream)
            reps = 10
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                torch.cuda._sleep(40_000_000)
            e0.record(stream)
            for _ in range(reps):
                shl.shl_field(h, d, r, F, gF, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            flops = 2.0 * 4 * (2 * d.K + 1) * r ** 3
            rows.append({"r": r, "charges": n, "ms": ms, "paper_h200_ms": FIELD_PAPER_H200_MS[(r, n)],
                         "fp64_gflops": flops / ms / 1e6, "out_gbs": 32.0 * r ** 3 / ms / 1e6})
    last = rows[-1]
    line = {"metric": "field evaluation time, F and grad F (r=256, 2N=256)", "value": last["ms"], "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "field (paper Table 1 shapes)", "K": 3},
            "roofline": {"bound": "fp64", "achieved": last["fp64_gflops"], "peak": fp64_peak,
                         "unit": "GFLOP/s", "frac": last["fp64_gflops"] / fp64_peak,
                         "peak_kind": "measured (shl_probe_peaks: FP64 FMA throughput)", "traffic": None,
                         "nominal_peak": FP64_NOMINAL_GFLOPS},
            "shapes": rows}
    print(json.dumps(line), flush=True)


def cubic_symmetry_err(C):
    """Largest deviation of C^H from cubic symmetry (C11=C22=C33, C12=C13=C23,
    C44=C55=C66, all other entries zero), relative to max |C|."""
    s = np.abs(C).max()
    dev = [C[0, 0] - C[1, 1], C[0, 0] - C[2, 2], C[0, 1] - C[0, 2], C[0, 1] - C[1, 2], C[3, 3] - C[4, 4],
           C[3, 3] - C[5, 5]]
    cubic = {(i, j) for i in range(3) for j in range(3)} | {(3, 3), (4, 4), (5, 5)}
    dev += [C[i, j] for i in range(6) for j in range(6) if (i, j) not in cubic]
    return float(np.max(np.abs(dev)) / s)


def run_grad(args):
    """Inverse-design gradients: a batch of designs at 64^3 (24 balanced
    charges, 10 % solid), objective E = sum (C^H - C_t)^2 with C_t isotropic
    (bulk 0.05, shear 0.02); forward and backward through the
    torch.autograd.Function over the adjoint (smoothed density, FP32 + FP64
    refinement at --tol; the backward starts from the forward's displacements).
    The thickness of each design is selected from its volume fraction first
    and then held fixed.  Accuracy: the first design's gradient against the
    FP64 path at 1e-12."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    from paper_2511_04025_b300.autograd import HomogenizeFn
    torch.cuda.set_device(0)
    r, batch, warm = 64, args.batch, 2
    designs = [inputs.gradient_64(1000 + i) for i in range(batch + warm)]
    Ct = torch.tensor(inputs.isotropic_target())
    o = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=args.tol, density=shl.SHL_SMOOTH)
    with shl.Context(0) as ctx:
        h = ctx.handle
        ts = [shl.shl_voxelize(h, d, r)["t"] for d in designs]

        def one(d, t):
            pos = torch.tensor(d.pos, requires_grad=True)
            q = torch.tensor(d.q, requires_grad=True)
            iso = torch.tensor(d.iso, dtype=torch.float64, requires_grad=True)
            tt = torch.tensor(t, dtype=torch.float64, requires_grad=True)
            C = HomogenizeFn.apply(pos, q, iso, tt, h, r, d.K, None, o)
            loss = ((C - Ct) ** 2).sum()
            loss.backward()
            return C.detach().numpy(), pos.grad.numpy(), q.grad.numpy(), float(tt.grad)

        for k in range(warm):
            one(designs[k], ts[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = [one(designs[warm + k], ts[warm + k]) for k in range(batch)]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        d0, t_0 = designs[warm], ts[warm]
        o64 = shl.default_solve_opts(precision=shl.SHL_FP64, tol=1e-12, density=shl.SHL_SMOOTH)
        C64 = shl.shl_homogenize(h, d0.copy(t=t_0), r, o64)[0]
        ref = shl.shl_grad(h, d0, r, o64, 2.0 * (C64 - Ct.numpy()), t=t_0)
    C0, gp, gq, gt = outs[0]
    scale = max(np.abs(ref["g_pos"]).max(), np.abs(ref["g_q"]).max(), abs(ref["g_t"]))
    gerr = max(np.abs(gp - ref["g_pos"]).max(), np.abs(gq - ref["g_q"]).max(), abs(gt - ref["g_t"])) / scale
    line = {"metric": "inverse-design gradients/sec (64^3, forward + adjoint through autograd)",
            "value": batch / wall, "unit": "gradients/s", "n_gpus": 1, "steps": batch, "warmup": warm,
            "ms_per_step": 1e3 * wall / batch, "higher_is_better": True, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": "gradient64", "designs": batch, "charges": 24, "vf": 0.10, "tol": args.tol,
                       "density": "smooth (logistic, kappa = ln 9 r)"},
            "accuracy": {"grad_rel_err": float(gerr), "reference": "FP64 GPU path, tol 1e-12 (first design)"},
            "e2e": {"value": batch / wall, "unit": "gradients/s", "note": "host wall clock, per-design sync"}}
    print(json.dumps(line), flush=True)


def run_design(args):
    """The inverse-design driver (Sec. 4.3 alternating scheme) at 64^3 on one
    design: maximise K_eff / V at 10 % solid, starting from 24 balanced
    charges.  Each outer iteration: thickness from the volume fraction,
    --alpha-steps Adam steps on alpha (forward + adjoint, smoothed density,
    FP32 + FP64 refinement at --tol), then --generations CMA-ES generations of
    --popsize candidates on the positions, each generation submitted at once
    to the serving path.  value = candidate evaluations per second over the
    timed outer iterations; the objective and K_eff as a fraction of the
    Hashin-Shtrikman upper bound are reported before and after."""
    import torch
    from paper_2511_04025_b300 import inputs, objectives, shl
    from paper_2511_04025_b300.design import InverseDesign
    torch.cuda.set_device(0)
    r, vf = args.r or 64, 0.10
    d = inputs.gradient_64(7)
    with shl.Context(0, max_batch=args.slots) as ctx:
        drv = InverseDesign(ctx.handle, d, r, args.objective, vf, popsize=args.popsize, seed=0, tol=args.tol)
        v0 = drv.value
        drv.run(1, 1, 1)  # warm-up: graphs, workspaces, serving slots
        ev0 = drv.hist.evaluations
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ta = tp = 0.0
        for _ in range(args.steps):
            a0 = time.perf_counter()
            drv.alpha_steps(args.alpha_steps)
            a1 = time.perf_counter()
            drv.position_generations(args.generations)
            tp += time.perf_counter() - a1
            ta += a1 - a0
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        evals = drv.hist.evaluations - ev0
        C, _ = shl.shl_homogenize(ctx.handle, drv.design, r, drv.opts)
    ku, gu = objectives.hs_upper(vf)
    keff = float(objectives.bulk_hill(torch.tensor(C, dtype=torch.float64)))
    gens = args.steps * args.generations
    line = {"metric": "inverse-design candidate evaluations/sec (64^3, CMA-ES positions through serving + Adam on alpha)",
            "value": evals / wall, "unit": "designs/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": "design64", "objective": args.objective, "vf": vf, "charges": 24, "r": r,
                       "alpha_steps": args.alpha_steps, "generations": args.generations, "popsize": drv.popsize_used,
                       "tol": args.tol, "slots": args.slots},
            "cma_candidates_per_s": gens * drv.popsize_used / tp, "alpha_steps_per_s": args.steps * args.alpha_steps / ta,
            "objective": {"start": v0, "end": drv.value, "trajectory": drv.hist.objective},
            "keff_frac_hs": keff / ku, "hs_upper": {"K": ku, "G": gu}}
    print(json.dumps(line), flush=True)


def solver_summary(stats):
    """Iterations (largest of the six load cases) and reliable updates per
    design: quartiles over the timed designs and the first 20 in order."""
    it = np.array([max(s["iters"]) for s in stats])
    nr = np.array([s["n_refine"] for s in stats])
    q = lambda v: {"min": int(v.min()), "median": float(np.median(v)), "max": int(v.max())}
    return {"iters_max": q(it), "n_refine": q(nr), "iters_max_first20": it[:20].tolist(),
            "relres_max": max(max(s["relres"]) for s in stats), "designs": len(stats)}


def bench_cubic128(h, stream, flush, opts, n=3, nb=8):
    """128^3 O_h designs (48 charges, 5 % solid): throughput of nb designs
    solved concurrently through shl_homogenize_batch (as the headline's
    batches), and n designs one at a time (single-design latency); CUDA
    events on the launch stream with L2 flushed before each timed region;
    C^H of seed 0 against the oracle's stored 128^3 value (tests/golden,
    solved to 1e-11) and the cubic symmetry of every C^H."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    r = 128
    designs = [inputs.cubic_128(s) for s in range(n + 1)]
    shl.shl_homogenize(h, designs[n], r, opts, stream=stream)  # warm-up (graphs, workspaces)
    batch = [inputs.cubic_128(100 + s) for s in range(nb)]
    shl.shl_homogenize_batch(h, batch[:2], [r] * 2, opts, stream=stream)  # warm-up of the slots
    with torch.cuda.stream(stream):
        flush.add_(1.0)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    Cb, stb = shl.shl_homogenize_batch(h, batch, [r] * nb, opts, stream=stream)
    b1.record(stream)
    stream.synchronize()
    batch_s = b0.elapsed_time(b1) / 1e3
    ms, Cs, its = [], [], []
    for d in designs[:n]:
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C, st = shl.shl_homogenize(h, d, r, opts, stream=stream)
        e1.record(stream)
        stream.synchronize()
        ms.append(e0.elapsed_time(e1))
        Cs.append(C)
        its.append(max(st["iters"]))
    out = {"designs_per_s": nb / batch_s, "designs": nb, "batch": f"{nb} designs concurrently",
           "iters_max_batch": [max(st["iters"]) for st in stb],
           "sequential": {"designs_per_s": n / (sum(ms) / 1e3), "ms_per_design": float(np.mean(ms)), "designs": n,
                          "iters_max": its},
           "cubic_symmetry_err_max": max(cubic_symmetry_err(C) for C in Cs + list(Cb))}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "cubic128_s0.json")) as f:
            g = np.array(json.load(f)["C"])
        out["chom_entry_err_vs_oracle"] = float(np.max(np.abs(Cs[0] - g) / np.maximum(np.abs(g), 1e-2 * np.abs(g).max())))
        out["oracle"] = "cubic_128 seed 0, oracle PCG to 1e-11"
    except OSError:
        out["chom_entry_err_vs_oracle"] = None
    return out


def bench_active(h, stream, flush, opts, n=10):
    """The active-set solve (Sec. 4.2.1: void culled, no ersatz floor) on 64^3
    throughput designs, one at a time, CUDA events on the launch stream, L2
    flushed between designs; seed 0's C^H against the oracle's active-set
    value and, as the model gap, against the oracle's ersatz-void value."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    r = 64
    o = shl.default_solve_opts(precision=opts.precision, tol=opts.tol, active=1)
    designs = [inputs.gaussian_64(s) for s in range(n + 1)]
    shl.shl_homogenize(h, designs[n], r, o, stream=stream)  # warm-up
    ms, its, Cs = [], [], []
    for d in designs[:n]:
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C, st = shl.shl_homogenize(h, d, r, o, stream=stream)
        e1.record(stream)
        stream.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(max(st["iters"]))
        Cs.append(C)

    def err(C, name):
        try:
            with open(os.path.join(ROOT, "tests", "golden", name + ".json")) as f:
                g = np.array(json.load(f)["C"])
        except OSError:
            return None
        return float(np.max(np.abs(C - g) / np.maximum(np.abs(g), 1e-2 * np.abs(g).max())))
    return {"designs_per_s": n / (sum(ms) / 1e3), "ms_per_design": float(np.mean(ms)), "designs": n,
            "iters_max": its, "tol": opts.tol,
            "chom_entry_err_vs_oracle_active": err(Cs[0], "gaussian64_s0_active"),
            "model_gap_vs_ersatz_oracle": err(Cs[0], "gaussian64_s0")}


# Timing table of the paper (Sec. 5.4, half-thickness t = 0.02): per r, the
# reported active voxels and total time per homogenisation on an H200 with its
# selective multigrid at the solver's default tolerance (context, not a target).
TABLE2_PAPER = {64: (32_000, 126.4), 128: (212_000, 182.9), 256: (1_500_000, 355.7)}


def bench_table2(h, stream, flush, opts, seeds=(0, 1)):
    """The timing table's setting: thin shells (t = 0.02, 32 charges) at r = 64,
    128 and 256 with the active set (Sec. 4.2.1), FP32 + refinement to --tol,
    one design at a time, CUDA events around the whole C-ABI call (field,
    voxelisation, six cell problems, C^H), L2 flushed between designs."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    o = shl.default_solve_opts(precision=opts.precision, tol=opts.tol, active=1)
    out = {}
    for r, (paper_active, paper_ms) in TABLE2_PAPER.items():
        shl.shl_homogenize(h, inputs.shell_256(len(seeds)), r, o, stream=stream)  # warm-up
        ms, its, act = [], [], []
        for sd in seeds:
            with torch.cuda.stream(stream):
                flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = shl.shl_homogenize(h, inputs.shell_256(sd), r, o, stream=stream)
            e1.record(stream)
            stream.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(max(st["iters"]))
            act.append(int(st["n_solid"]))
        out[str(r)] = {"ms_per_design": float(np.mean(ms)), "ms": ms, "iters_max": its, "active_voxels": act,
                       "paper_h200_ms": paper_ms, "paper_active_voxels": paper_active}
        torch.cuda.empty_cache()
    out["tol"] = opts.tol
    out["note"] = ("paper: H200, its own designs and the solver's default tolerance (5 V-cycles); "
                   "here: synthetic shells, relative residual <= tol")
    return out


def _golden(name):
    try:
        with open(os.path.join(ROOT, "tests", "golden", name + ".json")) as f:
            return json.load(f)
    except OSError:
        return None


def _entry_err(C, Cref):
    Cref = np.asarray(Cref)
    return float(np.max(np.abs(C - Cref) / np.maximum(np.abs(Cref), 1e-2 * np.abs(Cref).max())))


def bench_plain32(h, stream, n=3):
    """The plain method of the first configuration: 32^3, 8 charges +-1, 15 %
    solid, FP64 PCG to a relative residual of 1e-10, with the FP32 multigrid
    V-cycle as preconditioner (the default) and with point Jacobi; seed 0's
    C^H against the oracle's (solved to 1e-12)."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    g = _golden("plain32_s0")

    def run(precond):
        o = shl.default_solve_opts(precision=shl.SHL_FP64, tol=1e-10, precond=precond)
        shl.shl_homogenize(h, inputs.plain_32(n), 32, o, stream=stream)  # warm-up
        ms, Cs, its = [], [], []
        for sd in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            C, st = shl.shl_homogenize(h, inputs.plain_32(sd), 32, o, stream=stream)
            e1.record(stream)
            stream.synchronize()
            ms.append(e0.elapsed_time(e1))
            Cs.append(C)
            its.append(max(st["iters"]))
        return {"designs_per_s": n / (sum(ms) / 1e3), "ms_per_design": float(np.mean(ms)), "iters_max": its,
                "chom_entry_err_vs_oracle": _entry_err(Cs[0], g["C"]) if g else None}
    out = run(shl.SHL_PRECOND_MG)
    out.update({"designs": n, "precision": "fp64", "tol": 1e-10, "precond": "multigrid (FP32 V-cycle)",
                "jacobi": run(shl.SHL_PRECOND_JACOBI)})
    return out


def bench_grad64(h, stream, n=8):
    """Inverse-design gradients at 64^3 (the fifth configuration): n designs,
    24 charges +-1, 10 % solid, smoothed density, FP32 + refinement at tol
    1e-10, dE/dC^H = 2 (C^H - C^T); forward and adjoint through shl_grad.
    Seed 0 with the stored dE/dC^H against the oracle's gradient (every
    parameter, relative to the largest entry)."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    o = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=1e-10, density=shl.SHL_SMOOTH)
    Ct = inputs.isotropic_target()
    g = _golden("gradient64_s0")
    ts = [shl.shl_voxelize(h, inputs.gradient_64(sd), 64, stream=stream)["t"] for sd in range(n)]
    u = torch.empty(18 * 64 ** 3, dtype=torch.float64, device="cuda")
    shl.shl_grad(h, inputs.gradient_64(0), 64, o, np.zeros((6, 6)), u=u, t=ts[0], stream=stream)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sd in range(n):
        d = inputs.gradient_64(sd)
        fwd = shl.shl_grad(h, d, 64, o, np.zeros((6, 6)), u=u, t=ts[sd], stream=stream)
        ob = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=1e-10, density=shl.SHL_SMOOTH, warm_start=1)
        shl.shl_grad(h, d, 64, ob, 2.0 * (fwd["C"] - Ct), u=u, t=ts[sd], want_alpha=True, stream=stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    err = None
    if g:
        out = shl.shl_grad(h, inputs.gradient_64(0), 64, o, np.array(g["dEdC"]), t=g["t"], want_alpha=True,
                           stream=stream)
        scale = max(np.abs(g["g_pos"]).max(), np.abs(g["g_q"]).max(), abs(g["g_iso"]), abs(g["g_t"]),
                    np.abs(g["g_alpha"]).max())
        err = max(np.abs(out["g_pos"] - np.array(g["g_pos"])).max(), np.abs(out["g_q"] - np.array(g["g_q"])).max(),
                  abs(out["g_iso"] - g["g_iso"]), abs(out["g_t"] - g["g_t"]),
                  np.abs(out["g_alpha"] - np.array(g["g_alpha"])).max()) / scale
    return {"gradients_per_s": n / wall, "ms_per_gradient": 1e3 * wall / n, "designs": n, "tol": 1e-10,
            "clock": "host wall clock around forward + adjoint (each returns its results to the host)",
            "grad_rel_err_vs_oracle": None if err is None else float(err)}


def bench_field256(h, stream):
    """Field evaluation on the largest shape of the paper's field-timing table
    (r = 256, 2N = 256 charges): F and grad F in FP64, CUDA events."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    d = inputs.random_design(7, 256, 0.1)
    F = torch.empty(256 ** 3, dtype=torch.float64, device="cuda")
    gF = torch.empty(256 ** 3, 3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        shl.shl_field(h, d, 256, F, gF, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        shl.shl_field(h, d, 256, F, gF, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    del F, gF
    return {"ms": ms, "r": 256, "charges": 256, "paper_h200_ms": FIELD_PAPER_H200_MS[(256, 256)],
            "fp64_gflops": 2.0 * 4 * 7 * 256 ** 3 / ms / 1e6}


def bench_serve_short(args, n_requests=128):
    """A serving pass on the serving workload's mix (the Poisson stream of
    --serve, n_requests of it): burst throughput X, then Poisson arrivals at
    0.7 X; p50/p99 latency (submit -> result) overall and at 64^3."""
    import torch
    from paper_2511_04025_b300 import inputs, shl
    reqs = inputs.serving_stream(seed=0, n_requests=n_requests, rate_hz=1.0)
    opts = lambda warm: shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=args.tol, warm_start=int(warm))

    def replay(ctx, scale):
        t0 = time.perf_counter()
        tickets = []
        for q in reqs:
            if scale is not None:
                wait = q.t_arrive * scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            tickets.append((q, shl.shl_serve_submit(ctx.handle, q.design, q.r, opts(q.follow_up_of >= 0),
                                                    session=q.session)))
        out = [(q, shl.shl_serve_wait(ctx.handle, t)) for q, t in tickets]
        return time.perf_counter() - t0, out

    with shl.Context(0, max_batch=args.slots) as ctx:
        for r in (32, 64, 96):
            shl.shl_serve_wait(ctx.handle, shl.shl_serve_submit(ctx.handle, reqs[0].design, r, opts(False)))
        torch.cuda.synchronize()
        wall1, res1 = replay(ctx, None)
        X = len(reqs) / wall1
        span = reqs[-1].t_arrive if reqs[-1].t_arrive > 0 else 1.0
        wall2, res2 = replay(ctx, (len(reqs) / (0.7 * X)) / span)

    def lat(res, r=None):
        v = [x["t_done"] - x["t_submit"] for q, x in res if r is None or q.r == r]
        return (float(np.percentile(v, 50)), float(np.percentile(v, 99))) if v else (None, None)
    p50, p99 = lat(res2)
    p50_64, p99_64 = lat(res2, 64)
    return {"requests": len(reqs), "slots": args.slots, "burst_designs_per_s": X,
            "poisson_designs_per_s": len(reqs) / wall2, "latency_s": {"p50": p50, "p99": p99, "p50_64": p50_64,
                                                                      "p99_64": p99_64},
            "all_converged": all(x["stats"]["status"] == 0 for _, x in res1 + res2),
            "mix": "32/64/96^3 @ .50/.35/.15, 8-64 charges, 3-20 % solid, 25 % warm-start follow-ups"}


def run_serve(args):
    """Serving workload: a Poisson request stream (grids 32^3/64^3/96^3 at
    0.50/0.35/0.15, 8-64 charges, 3-20 % solid, 25 % warm-start follow-ups).
    Pass 1 submits everything at once (saturating burst) and measures the
    closed-loop throughput X; pass 2 replays the stream with Poisson arrivals at
    0.7 X.  Latency = submit -> result."""
    import torch
    from paper_2511_04025_b300 import inputs, shl

    torch.cuda.set_device(0)
    reqs = inputs.serving_stream(seed=0, n_requests=args.requests, rate_hz=1.0)
    opts = lambda warm: shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=args.tol, warm_start=int(warm))

    def replay(ctx, scale):
        t0 = time.perf_counter()
        tickets = []
        for q in reqs:
            if scale is not None:
                wait = q.t_arrive * scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            warm = q.follow_up_of >= 0
            tickets.append((q, shl.shl_serve_submit(ctx.handle, q.design, q.r, opts(warm), session=q.session)))
        out = [(q, shl.shl_serve_wait(ctx.handle, t)) for q, t in tickets]
        wall = time.perf_counter() - t0
        return wall, out

    with shl.Context(0, max_batch=args.slots) as ctx:
        # warm-up: one design per grid size
        for r in (32, 64, 96):
            shl.shl_serve_wait(ctx.handle, shl.shl_serve_submit(ctx.handle, reqs[0].design, r, opts(False)))
        torch.cuda.synchronize()
        with ClockSampler(0) as clk1:
            wall1, res1 = replay(ctx, None)
        X = len(reqs) / wall1
        span = reqs[-1].t_arrive if reqs[-1].t_arrive > 0 else 1.0
        scale = (len(reqs) / (0.7 * X)) / span  # seconds of replay per unit of stream time
        c0 = shl.shl_get_counters(ctx.handle)["kernel_launches"]
        with ClockSampler(0) as clk2:
            wall2, res2 = replay(ctx, scale)
        c1 = shl.shl_get_counters(ctx.handle)["kernel_launches"]

    def lat(res, r=None):
        v = [x["t_done"] - x["t_submit"] for q, x in res if r is None or q.r == r]
        return (float(np.percentile(v, 50)), float(np.percentile(v, 99))) if v else (None, None)

    ok = all(x["stats"]["status"] == 0 for _, x in res1 + res2)
    failures = [{"pass": ps, "r": q.r, "status": x["stats"]["status"], "warm": x["warm"], "slot": x["slot"],
                 "iters_max": max(x["stats"]["iters"]), "relres_max": max(x["stats"]["relres"])}
                for ps, res in (("burst", res1), ("poisson", res2)) for q, x in res if x["stats"]["status"] != 0]
    p50, p99 = lat(res2)
    p50_64, p99_64 = lat(res2, 64)
    line = {
        "metric": "served designs/sec (Poisson arrivals at 0.7x burst throughput)", "value": len(reqs) / wall2,
        "unit": "designs/s", "n_gpus": 1, "steps": len(reqs), "warmup": 3, "ms_per_step": 1e3 * wall2 / len(reqs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "serve", "requests": len(reqs), "slots": args.slots, "grids": "32/64/96 @ .50/.35/.15",
                   "tol": args.tol, "warm_start_share": float(np.mean([q.follow_up_of >= 0 for q in reqs]))},
        "latency_s": {"p50": p50, "p99": p99, "p50_64": p50_64, "p99_64": p99_64},
        "burst": {"designs_per_s": X, "latency_p50": lat(res1)[0], "latency_p99": lat(res1)[1]},
        "warm_hits": int(sum(1 for _, x in res2 if x["warm"])), "all_converged": ok,
        "failures": failures[:16],
        "clocks": clk2.summary(), "gpu_launches": int(c1 - c0),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="shl", choices=["shl", "reference"])
    ap.add_argument("--workload", default="gaussian64", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="fp32r", choices=["fp32r", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the sub-records (128^3, serving, active set, ...)")
    ap.add_argument("--active", action="store_true",
                    help="solve the active-set problem (void culled, no ersatz floor) instead of the ersatz one")
    ap.add_argument("--tol", type=float, default=1e-7,
                    help="relative residual of the cell problems (the metric asks C^H within 1e-4; 1e-7 gives <= 4e-7)")
    ap.add_argument("--serve", action="store_true", help="serving workload (Poisson stream) instead of the bench")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--kernel", choices=["apply"], help="time the dominant kernel alone instead of the bench")
    ap.add_argument("--field", action="store_true", help="field throughput on the paper's Table 1 shapes")
    ap.add_argument("--grad", action="store_true", help="inverse-design gradients on a batch of 64^3 designs")
    ap.add_argument("--batch", type=int, default=64, help="designs per gradient batch (--grad)")
    ap.add_argument("--batch-designs", type=int, default=16,
                    help="designs per timed step, solved concurrently on the serving slots through "
                         "shl_homogenize_batch (1: one at a time).  On the same 32 64^3 designs: 16.9 designs/s one "
                         "at a time, 19.7 at 4 or 8, 20.4 at 16, 20.1 at 32")
    ap.add_argument("--design", action="store_true", help="inverse-design driver at 64^3 (Keff by default)")
    ap.add_argument("--objective", default="Keff", choices=["Ex", "Cavg", "Keff", "Geff", "coupling", "isotropy"])
    ap.add_argument("--alpha-steps", type=int, default=4)
    ap.add_argument("--generations", type=int, default=4)
    ap.add_argument("--popsize", type=int, default=16)
    ap.add_argument("--r", type=int, default=0, help="grid size for --kernel (default: the workload's)")
    ap.add_argument("--launches", type=int, default=40, help="timed launches for --kernel")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return run_kernel(args)
    if args.field:
        return run_field(args)
    if args.grad:
        return run_grad(args)
    if args.design:
        return run_design(args)
    if args.serve:
        return run_serve(args)

    import torch
    from paper_2511_04025_b300 import inputs, shl

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    gen, r, desc = WORKLOADS[args.workload]
    prec = shl.SHL_FP32_REFINE if args.precision == "fp32r" else shl.SHL_FP64
    opts = shl.default_solve_opts(precision=prec, tol=args.tol, active=int(args.active))
    ctx = shl.Context(local, max_batch=args.slots)
    h = ctx.handle
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 126 MB L2
    B = max(1, args.batch_designs)
    designs = [getattr(inputs, gen)(sd) for sd in rank_seeds(rank, (args.warmup + args.steps) * B)]
    batches = [designs[k * B:(k + 1) * B] for k in range(args.warmup + args.steps)]

    def solve(batch):
        """One step: a batch of designs through the public batch entry point
        (concurrent on the serving slots), or one design alone for B = 1."""
        if len(batch) == 1:
            C, st = shl.shl_homogenize(h, batch[0], r, opts, stream=stream)
            return [C], [st]
        C, st = shl.shl_homogenize_batch(h, batch, [r] * len(batch), opts, stream=stream)
        return list(C), st

    for k in range(args.warmup):
        solve(batches[k])
    torch.cuda.synchronize()
    c0 = shl.shl_get_counters(h)["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall = []
    stats = []
    Cs = []
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.add_(1.0)  # L2 flush between timed steps (untimed)
            stream.synchronize()
            t0 = time.perf_counter()
            ev[k][0].record(stream)
            C, st = solve(batches[args.warmup + k])
            Cs += C
            ev[k][1].record(stream)
            stream.synchronize()
            wall.append(time.perf_counter() - t0)
            stats += st
    torch.cuda.synchronize()
    c1 = shl.shl_get_counters(h)["kernel_launches"]
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    wall_s = sum(wall)
    dev_s, wall_s = max_over_ranks(world, dev_s, wall_s)
    value = job_rate(world, args.steps, B, dev_s)
    e2e = job_rate(world, args.steps, B, wall_s)

    # the same designs one at a time (single-design latency), a sample of them
    seq = None
    if B > 1:
        n_seq = min(len(Cs), 8)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(n_seq):
            shl.shl_homogenize(h, designs[args.warmup * B + i], r, opts, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_s = e0.elapsed_time(e1) / 1e3
        seq = {"designs_per_s": n_seq / seq_s, "ms_per_design": 1e3 * seq_s / n_seq, "designs": n_seq}

    # dominant kernel: the FP32 stiffness apply of the inner solves, timed on
    # the launch stream on the last design's mask
    apply_s = time_apply(h, r, designs[-1], stream)
    roofline = apply_roofline(r, apply_s)
    arith_peaks = shl.shl_probe_peaks(h)

    # accuracy of the timed designs (untimed): C^H against the plain FP64 GPU
    # path solved to 1e-11, entry error relative to max(|C_ij|, 1e-2 max|C|);
    # every design of the first timed batch and the first of each later one
    ref = shl.default_solve_opts(precision=shl.SHL_FP64, tol=1e-11, active=int(args.active))
    ref_desc = ("FP64 GPU path (FP64 CG, FP32 multigrid preconditioner), tol 1e-11"
                + (", same active set" if args.active else ""))
    if r >= 256:  # the FP64 mode (point Jacobi) takes minutes per design here
        ref = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=1e-10, active=int(args.active))
        ref_desc = "same path at tol 1e-10 (self-consistency; no FP64 reference at 256^3)"
    acc = 0.0
    check = list(range(min(B, 8))) + [k * B for k in range(1, args.steps)]
    Crs, _ = shl.shl_homogenize_batch(h, [designs[args.warmup * B + i] for i in check], [r] * len(check), ref,
                                      stream=stream)
    for i, Cr in zip(check, Crs):
        acc = max(acc, float(np.max(np.abs(Cs[i] - Cr) / np.maximum(np.abs(Cr), 1e-2 * np.abs(Cr).max()))))
    (acc,) = max_over_ranks(world, acc)
    accuracy = {"chom_entry_err_max": acc, "bound": 1e-4, "designs": len(check) * world, "reference": ref_desc}
    if args.workload == "cubic128":
        accuracy["cubic_symmetry_err_max"] = max(cubic_symmetry_err(C) for C in Cs)

    # precision at equal accuracy: one design (the first timed one) alone on
    # the same GPU, solved to the same tolerance by the plain FP64 path
    # (point-Jacobi PCG), by FP32 + refinement with the same point-Jacobi
    # preconditioner, and by FP32 + refinement with the multigrid
    compare = None
    if not args.no_compare and prec == shl.SHL_FP32_REFINE and rank == 0:
        d_first = batches[args.warmup][0]

        def alone(o):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st_ = shl.shl_homogenize(h, d_first, r, o, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3, max(st_["iters"])
        jac = shl.SHL_PRECOND_JACOBI
        s64, it64 = alone(shl.default_solve_opts(precision=shl.SHL_FP64, tol=args.tol, precond=jac))
        s64m, it64m = alone(shl.default_solve_opts(precision=shl.SHL_FP64, tol=args.tol))
        s32j, it32j = alone(shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=args.tol, precond=jac))
        s32m, it32m = alone(opts)
        compare = {"fp64_designs_per_s": 1.0 / s64, "fp64_iters_max": it64, "fp64_precond": "jacobi",
                   "fp32r_jacobi_designs_per_s": 1.0 / s32j, "fp32r_jacobi_iters_max": it32j,
                   "same_precond_ratio": s64 / s32j,
                   "fp64_mg_designs_per_s": 1.0 / s64m, "fp64_mg_iters_max": it64m,
                   "fp32r_mg_designs_per_s": 1.0 / s32m, "fp32r_mg_iters_max": it32m,
                   "same_precond_ratio_mg": s64m / s32m, "tol": args.tol, "designs": 1,
                   "note": "one design alone, same tolerance; same_precond_ratio = FP32 + refinement over FP64 "
                           "with point-Jacobi PCG on both, same_precond_ratio_mg the same with the FP32 "
                           "multigrid V-cycle preconditioning both"}

    # the rest of the metric: designs/s at 128^3 (O_h designs, C^H against the
    # oracle's 128^3 value and cubic symmetry) and served p50/p99 latency
    sub128 = serve = active = plain32 = grad64 = field256 = table2 = None
    if rank == 0 and world == 1 and args.workload == "gaussian64" and not args.no_extra:
        sub128 = bench_cubic128(h, stream, flush, opts)
        active = bench_active(h, stream, flush, opts)
        table2 = bench_table2(h, stream, flush, opts)
        plain32 = bench_plain32(h, stream)
        grad64 = bench_grad64(h, stream)
        field256 = bench_field256(h, stream)
        serve = bench_serve_short(args, n_requests=512)  # the serving workload's 512 requests

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, per, sample, cores = oracle_sample(designs[0], r, golden_iters(args.workload))
        cpu = {"value": v, "unit": "designs/s", "cores": cores, "kind": "oracle", "sample": sample,
               "extrapolated": True, "validation": oracle_validate()}

    if rank == 0:
        d0 = designs[args.warmup]
        line = {
            "metric": "homogenized designs/sec", "value": value, "unit": "designs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
            "designs_per_step": B, "sequential": seq,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": bench_config(args, r, desc, world),
            "e2e": {"value": e2e, "unit": "designs/s", "h2d_bytes_per_step": int(B * (d0.pos.nbytes + d0.q.nbytes)),
                    "d2h_bytes_per_step": B * 36 * 8},
            "roofline": roofline, "arith_peaks_gflops": arith_peaks, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": int(c1 - c0),
            "solver": solver_summary(stats),
            "accuracy": accuracy, "compare": compare, "cubic128": sub128, "active_set": active, "serve": serve,
            "plain32_fp64": plain32, "grad64": grad64, "field256": field256, "table2": table2,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
