"""Benchmark of the subspace-construction hot path on GB300.

The default workload is the largest single-GPU configuration: the splat-like
cloud of 1,000,000 points (a mixture of 64 anisotropic Gaussians, axis scales
log-uniform 0.02-0.3, volumes from the 16-nearest-neighbour density, E
log-uniform 1e4-1e7 per Gaussian, nu = 0.45) through the paper's own route for
splats: the points themselves are the quadrature points, K = 1,000 kernel
centres are chosen among them by farthest-point sampling, Gaussian kernels of
radius the second-nearest-centre distance, cut at 3 r_k; k = 64 lowest modes
(the constant one included).  One step = rkpm_build_twoset +
assemble_hessian + eigenmodes with the inputs already resident in HBM, L2
flushed (a 256 MB write) before every step, timed with CUDA events on the
library's stream with the profiler off except for the one kernel class whose
roofline is reported.  `value` is the time to k modes at relative residual
1e-6 (lower is better).

The same JSON line carries: `roofline` of the dominant kernel (algorithmic
bytes or operations over its CUDA-event duration inside the timed region),
`stage_ms_per_step` from a separate profiled pass, `e2e` through the C-ABI
host-buffer call (pinned host inputs copied in and the modes copied out
inside the timed region), `gpu_launches`, SM `clocks` sampled during the timed
region, `cpu_baseline` (the FP64 oracle timed on the host cores on a bounded
sample of the same workload, scaled to it), and `torus50k`: the nodal
discretisation on the 50,000-particle solid torus (k = 32), plain and from the
learned warm start, with the roofline of its preconditioner step, its fused
(H, M) block product and the skinning weight fields of its modes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload splat|torus|twoset-torus|batch] [--prec fp64|fp32]
                  [--tol T] [--cheb D] [--cheb-fp64 D] [--fp32-phase 0|1]
                  [--fp32-tol T] [--precond-tc 0|1] [--precond-compact 0|1]
                  [--no-cpu-baseline] [--no-torus]

`--workload torus` prints the torus line on its own (the nodal path alone);
`--workload twoset-torus` times the two-set construction on the torus as
49,584 inside-grid quadrature points (h = 0.02), K = 1,000, k = 32;
`--workload batch` times one eigenmodes_batched call on 32 objects of
2,000-200,000 particles per step (objects/s, particles/s).

With N > 1 (torchrun, one process per GPU) every rank solves its own object
(replicas: the path has no cross-GPU exchange; weak scaling) and the reported
time is the maximum over ranks.  `--impl reference` times the FP64 CPU oracle
on the host cores (rank 0 only) on the same workload and config: each step
times the oracle's stages on bounded samples and scales them to the whole
workload (see `oracle_splat_step`).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import atexit
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-k-modes at rel. residual 1e-6 (s), warm vs plain; SpMM HBM GB/s"

SPLAT = dict(n=1_000_000, K=1000, k=64, trunc=3.0, start=0)
SPLAT_WORKLOAD = (
    "splat-like cloud: 1,000,000 points from a mixture of 64 anisotropic Gaussians (seed 3, "
    "axis scales log-uniform 0.02-0.3), volumes from the 16-nearest-neighbour density, "
    "E log-uniform 1e4-1e7 per Gaussian, nu=0.45; two-set RKPM (the points as quadrature "
    "points, K=1,000 farthest-point centres, Gaussian kernels with r_k = 2nd-nearest-centre "
    "distance cut at 3 r_k); k=64 lowest modes incl. the constant mode")
TORUS_WORKLOAD = ("solid torus R=0.5 r=0.2, 50,000 particles rejection-sampled (seed 2), "
                  "cubic B-spline support 2.0x spacing, Neo-Hookean E=1e6 nu=0.4, "
                  "k=32 lowest modes incl. the constant mode")
TWOSET_TORUS_WORKLOAD = ("solid torus R=0.5 r=0.2 as 49,584 inside-grid quadrature points "
                         "(h=0.02), K=1,000 farthest-point centres, Gaussian kernels with "
                         "r_k = 2nd-nearest-centre distance cut at 3 r_k, Neo-Hookean E=1e6 "
                         "nu=0.4, k=32 lowest modes incl. the constant mode")
L2_NOTE = "flushed by a 256 MB write before every timed step"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "kind": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "kind": "fallback"}


def _traffic(cls, kernel):
    """DRAM bytes per launch from the committed ncu capture, if it was taken on
    this kernel (null once the kernel has changed)."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(cls)
    if e is None or e.get("kernel") != kernel:
        return None
    return e.get("bytes_per_launch")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region.

    Started before the warm-up steps (enter() returns at once when already
    started), so that nvidia-smi's own start-up overlaps untimed work; the
    samples then cover the warm-up and the timed steps."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        if self.proc:
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            atexit.register(self._kill)  # never left sampling if a step raises
        except Exception:
            self.proc = None
        return self

    def _kill(self):
        if self.proc and self.proc.poll() is None:
            self.proc.kill()

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# Per-workload defaults of the options a flag leaves unset.  The splat follows
# its configuration's precision plan: shape functions and tile sums in FP32
# (the matrices stored in FP64), FP32 preconditioner steps of degree 32 (16
# iterations instead of 21 at degree 16 on this K = 1,000 pencil; degrees 48
# to 96 gave no fewer), and the FP32 phase runs to 3e-5 before it hands over
# (its rounding floor is lower on this small pencil than on the 50k torus);
# the nodal torus keeps degree 16, the hand-over at 1e-4 and the double-float
# build of an FP64 context.
WORKLOAD_DEFAULTS = {
    "splat": dict(cheb=32, cheb_fp64=48, build_prec="fp32", fp32_tol=3e-5),
    "torus": dict(cheb=16, cheb_fp64=48, build_prec="fp64", fp32_tol=1e-4),
    "twoset-torus": dict(cheb=16, cheb_fp64=48, build_prec="fp64", fp32_tol=1e-4),
    "batch": dict(cheb=16, cheb_fp64=48, build_prec="fp64", fp32_tol=1e-4),
}


def _opt(args, name, workload=None):
    v = getattr(args, name, None)
    return WORKLOAD_DEFAULTS[workload or args.workload][name] if v is None else v


def _opts(args, workload=None):
    from paper_2605_29318_gb300 import binding
    return binding.default_opts(tol=args.tol, cheb_degree=_opt(args, "cheb", workload),
                                max_iter=args.max_iter, fp32_phase=args.fp32_phase,
                                cheb_degree_fp64=_opt(args, "cheb_fp64", workload),
                                precond_tc=args.precond_tc,
                                fp32_tol=_opt(args, "fp32_tol", workload),
                                precond_compact=args.precond_compact)


def _dtype_name(args, workload=None):
    if args.prec == "fp32":
        return "f32+bf16"
    solve = "f32+bf16, then f32x2 double-float" if args.fp32_phase else "f64"
    if (workload or args.workload) == "splat" and _opt(args, "build_prec", "splat") == "fp32":
        return "f32 build (f64 matrices); solve " + solve
    return solve


# ------------------------------------------------------------------ workloads
def splat_cloud():
    from paper_2605_29318_gb300 import synth
    return synth.gaussian_mixture(SPLAT["n"])


def splat_config(args):
    """The config object of the splat line (identical in both arms)."""
    return {"workload": SPLAT_WORKLOAD, "precision": args.prec,
            "build_precision": _opt(args, "build_prec", "splat"), "tol": args.tol,
            "cheb_degree": _opt(args, "cheb", "splat"),
            "cheb_degree_fp64": _opt(args, "cheb_fp64", "splat"),
            "fp32_tol": _opt(args, "fp32_tol", "splat"),
            "points": SPLAT["n"], "K": SPLAT["K"], "k": SPLAT["k"], "l2": L2_NOTE,
            "parallelism": "single GPU"}


def torus_config(args):
    return {"workload": TORUS_WORKLOAD, "precision": args.prec, "tol": args.tol,
            "cheb_degree": _opt(args, "cheb", "torus"),
            "cheb_degree_fp64": _opt(args, "cheb_fp64", "torus"), "n": 50000, "k": 32, "l2": L2_NOTE, "parallelism": "single GPU"}


def twoset_torus_config(args):
    return {"workload": TWOSET_TORUS_WORKLOAD, "precision": args.prec, "tol": args.tol,
            "points": 49584, "K": 1000, "k": 32, "l2": L2_NOTE, "parallelism": "single GPU"}


# ------------------------------------------------------------------ the oracle on host cores
class OracleSplat:
    """The FP64 oracle's two-set path on the splat workload, timed on a bounded
    sample and scaled to the whole workload.  Set-up (untimed): the cloud, and
    K = 1,000 farthest-point centres of a 100,000-point random subsample (for
    the per-point stages only: their covering counts match the full
    sampling's).  Each step times
      * farthest-point sampling of all 1,000,000 points for `fps_k` centres,
        scaled by (K - 1) / (fps_k - 1) (one pass over the points per centre);
      * the radii of the K centres (whole);
      * covering lists and Gaussian shape functions at `n_sample` random points,
        and their contribution to H_w and M (sparse products), scaled by
        n / n_sample (the work is per point);
      * the dense generalized eigensolve of the K x K pencil for k = 64
        (whole; the sample's volumes scaled by n / n_sample so that M is
        positive definite)."""

    def __init__(self, fps_k=40, n_sample=16000, seed=0):
        import numpy as np
        from oracle import twoset
        self.c = splat_cloud()
        self.fps_k = fps_k
        self.n_sample = n_sample
        rng = np.random.default_rng(seed)
        sub = rng.choice(self.c.n, 100_000, replace=False)
        cen = twoset.farthest_point_sampling(self.c.X[sub], SPLAT["K"])
        self.P = self.c.X[sub][cen]
        self.rng = rng

    def describe(self):
        return (f"FP64 oracle (farthest-point sampling, radii, Gaussian shape functions, "
                f"sparse H_w/M, dense eigensolve) on the splat workload: farthest-point "
                f"sampling of all {SPLAT['n']:,} points for {self.fps_k} centres scaled to "
                f"K={SPLAT['K']:,}; shape functions and H_w/M at {self.n_sample:,} random "
                f"points scaled to {SPLAT['n']:,}; radii and the K x K eigensolve whole")

    def step(self):
        import numpy as np
        from oracle import eigen, twoset
        c, K, k = self.c, SPLAT["K"], SPLAT["k"]
        n = c.n
        t0 = time.perf_counter()
        twoset.farthest_point_sampling(c.X, self.fps_k, SPLAT["start"])
        t1 = time.perf_counter()
        r = twoset.radii(self.P)
        t2 = time.perf_counter()
        pick = np.sort(self.rng.choice(n, self.n_sample, replace=False))
        Xs = c.X[pick]
        scale = n / self.n_sample
        ptr, idx, phi, dphi, _ = twoset.shape_functions(Xs, self.P, r, SPLAT["trunc"])
        H, M = twoset.assemble(Xs.shape[0], K, ptr, idx, phi, dphi,
                               c.v[pick].astype(np.float64) * scale, c.E[pick], c.nu)
        t3 = time.perf_counter()
        eigen.eigh_dense(H, M, k)
        t4 = time.perf_counter()
        est = ((t1 - t0) * (K - 1) / (self.fps_k - 1) + (t2 - t1) + (t3 - t2) * scale
               + (t4 - t3))
        return est, t4 - t0


def oracle_torus_step(n=10000, k=32):
    """The FP64 oracle's whole nodal path on a 10,000-particle sample of the
    torus (the 50,000-particle problem's shift-invert solve alone takes
    minutes): brute-force neighbours, shape functions, sparse H_w and M,
    shift-invert eigsh."""
    from oracle import assembly, eigen, rkpm
    from paper_2605_29318_gb300 import synth
    c = synth.torus(n, seed=2)
    t0 = time.perf_counter()
    ptr, idx = rkpm.neighbours(c.X, c.a, chunk=64)
    phi, dphi, _ = rkpm.shape_functions(c.X, c.a, ptr, idx)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam, C = eigen.eigsh_sparse(H, M, k)
    return time.perf_counter() - t0


def oracle_twoset_torus_step(h=0.02, K=1000, k=32):
    """The FP64 oracle's two-set path on the whole two-set torus workload."""
    from oracle import eigen, twoset
    from paper_2605_29318_gb300 import synth
    X, v = synth.torus_grid(h)
    t0 = time.perf_counter()
    _, _, H, M = twoset.build(X, v, K, 1e6, 0.4, trunc=3.0)
    eigen.eigh_dense(H, M, k)
    return time.perf_counter() - t0


def cpu_baseline_splat():
    o = OracleSplat()
    est, wall = o.step()
    return {"value": round(est, 3), "unit": "s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": o.describe() + f" ({wall:.1f} s of CPU work)"}


# ------------------------------------------------------------------ GPU runs
def _timed(step, st, flush):
    import torch
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    out = step()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def _roofline(kind, desc, work, unit_work, ms, cnt, peaks, traffic=None, extra=None):
    """roofline object: `work` algorithmic bytes (hbm) or FP32 operations (alu)
    per launch over the mean launch duration `ms`."""
    if not cnt:
        return None
    if kind == "hbm":
        achieved = work / (ms * 1e-3) / 1e9
        peak, unit = peaks["hbm_gbs"], "GB/s"
    else:
        achieved = work / (ms * 1e-3) / 1e12
        peak, unit = peaks["fp32_tflops"], "TFLOP/s"
    out = {"kernel": desc, "bound": kind, "achieved": round(achieved, 2), "peak": peak,
           "peak_kind": peaks["kind"], "unit": unit, "frac": round(achieved / peak, 4),
           "traffic": traffic, unit_work: work, "avg_launch_ms": round(ms, 5), "launches": cnt}
    if extra:
        out.update(extra)
    return out


def run_splat(args, ctx, dev, local):
    """The splat workload: device-timed steps (profiler on for the roofline
    kernel's class only), a profiled pass for the stage split, and e2e steps
    through the host-buffer C call."""
    import numpy as np
    import torch

    from paper_2605_29318_gb300 import binding
    c = splat_cloud()
    K, k, trunc, start = SPLAT["K"], SPLAT["k"], SPLAT["trunc"], SPLAT["start"]
    X = torch.from_numpy(c.X).to(dev)
    v = torch.from_numpy(c.v).to(dev)
    E = torch.from_numpy(np.ascontiguousarray(c.E, np.float32)).to(dev)
    nu = float(c.nu)
    opts = _opts(args, "splat")
    modes = torch.empty((k, K), dtype=ctx.dtype, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    if args.prec == "fp64":
        ctx.set_build_precision(_opt(args, "build_prec", "splat"))

    def step():
        ctx.rkpm_build_twoset(X, v, K, trunc, start)
        ctx.assemble_hessian(E, None, 1.0, nu)
        return ctx.eigenmodes(k, opts, modes_out=modes, check=False)

    clk = Clocks(local).__enter__()
    for _ in range(args.warmup):
        _timed(step, st, flush)
    roof_cls = "asm_values"
    ctx.profile(True, classes=[roof_cls])
    launches0 = binding.launch_count()
    times, reps = [], []
    with clk:
        for _ in range(args.steps):
            t, (_, _, rep, status) = _timed(step, st, flush)
            times.append(t)
            reps.append((rep, status))
    launches = binding.launch_count() - launches0
    roof_cnt, roof_tot = ctx.profile_read()[roof_cls]
    ctx.profile(False)
    # stage split from a separate profiled pass
    nprof = max(1, min(args.steps, 3))
    ctx.profile(True)
    for _ in range(nprof):
        _timed(step, st, flush)
    prof = ctx.profile_read()
    ctx.profile(False)
    n_, n1, n2 = ctx.sizes()
    # e2e: pinned host inputs in, the modes out, through ff_subspace_twoset_host
    Xp = torch.from_numpy(c.X).pin_memory()
    vp = torch.from_numpy(c.v).pin_memory()
    Ep = torch.from_numpy(np.ascontiguousarray(c.E, np.float32)).pin_memory()
    host_modes = torch.empty((k, K), dtype=ctx.dtype).pin_memory()
    e2e, h2d, d2h = [], 0, 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, h2d, d2h, _ = binding.subspace_twoset_from_host(
            Xp, vp, Ep, nu, K, k, trunc, start, args.prec, opts, local, ctx, host_modes)
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    ms = sum(times) / len(times)
    rep, status = reps[-1]
    return {"ms": ms, "times": times, "rep": rep, "status": status, "prof": prof,
            "nprof": nprof, "roof": (roof_cls, roof_cnt, roof_tot), "launches": launches,
            "clocks": clk.summary(), "sizes": (n_, n1, n2), "e2e_s": sum(e2e) / len(e2e),
            "h2d": h2d, "d2h": d2h}


def splat_line(args, r, peaks):
    n, n1, n2 = r["sizes"]
    cls, cnt, tot = r["roof"]
    ms_launch = tot / max(cnt, 1)
    # assembly of the K x K H_w and M from the two-set shape functions:
    # per quadrature point i with c_i covering centres, c_i^2 pair products,
    # each 4 multiply-adds (3 gradient components for H_w, 1 for M); the
    # double-float sums of FP64 contexts cost 12 FP32 operations per
    # multiply-add, the FP32 ones 2
    pair_products = r["pair_products"]
    df = args.prec == "fp64" and _opt(args, "build_prec", "splat") == "fp64"
    per_mac = 24 if df else 2
    ops = 4 * pair_products * per_mac
    kern = "k_tset_tiles" if df else "k_tset_tiles_once"
    roof = _roofline("alu", kern + " (two-set H_w and M: dense 64 x 64 register tiles of "
                     "24-point tiles grouped by nearest centre)",
                     ops, "algorithmic_fp32_ops_per_launch", ms_launch, cnt, peaks,
                     traffic=_traffic("asm_values", kern),
                     extra={"pair_products": pair_products,
                            "fp32_ops_per_multiply_add": per_mac // 2 * 2})
    line = {
        "metric": METRIC, "value": round(r["ms"] / 1000.0, 5), "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms"], 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype_name(args), "data": "synthetic", "config": splat_config(args),
        "sizes": {"K": n, "pairs": n1, "matrix_entries": n2},
        "roofline": roof,
        "stage_ms_per_step": {kk: round(vv[1] / r["nprof"], 3) for kk, vv in r["prof"].items()
                              if vv[0]},
        "solver": {"iterations": r["rep"]["iterations"],
                   "fp32_iterations": r["rep"]["fp32_iterations"], "status": r["status"],
                   "max_residual": r["rep"]["max_residual"]},
        "e2e": {"value": round(r["e2e_s"], 5), "unit": "s", "h2d_bytes_per_step": int(r["h2d"]),
                "d2h_bytes_per_step": int(r["d2h"]), "call": "ff_subspace_twoset_host"},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
    }
    return line


def run_torus(args, ctx, dev, local, rank, world):
    """The nodal 50,000-particle torus: plain and warm-start steps, the
    preconditioner step's roofline, the fused block product, e2e through the
    host-buffer call, the skinning weight fields of the modes."""
    import torch

    from paper_2605_29318_gb300 import binding, synth, train_warmstart
    c = synth.torus(50000, seed=2 + 1000 * rank)
    X = torch.from_numpy(c.X).to(dev)
    v = torch.from_numpy(c.v).to(dev)
    a = torch.from_numpy(c.a).to(dev)
    opts = _opts(args, "torus")
    net = binding.Net(local)
    net.set_params(train_warmstart.load_weights())
    modes = torch.empty((32, c.n), dtype=ctx.dtype, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step(warm=False):
        ctx.rkpm_build(X, v, a)
        ctx.assemble_hessian(None, None, c.E, c.nu)
        X0 = ctx.warmstart_block(net, 32, opts) if warm else None
        return ctx.eigenmodes(32, opts, X0=X0, modes_out=modes, check=False)

    clk = Clocks(local).__enter__()
    for _ in range(args.warmup):
        _timed(step, st, flush)
    ctx.profile(True, classes=["precond"])
    launches0 = binding.launch_count()
    times, reps = [], []
    with clk:
        for _ in range(args.steps):
            t, (_, _, rep, status) = _timed(step, st, flush)
            times.append(t)
            reps.append((rep, status))
    launches = binding.launch_count() - launches0
    pre_cnt, pre_tot = ctx.profile_read()["precond"]
    ctx.profile(False)
    nprof = max(1, min(args.steps, 3))
    ctx.profile(True)
    for _ in range(nprof):
        _timed(step, st, flush)
    prof = ctx.profile_read()
    ctx.profile(False)
    for _ in range(args.warmup):
        _timed(lambda: step(True), st, flush)
    wtimes, wreps = [], []
    for _ in range(args.steps):
        t, (_, _, rep, status) = _timed(lambda: step(True), st, flush)
        wtimes.append(t)
        wreps.append((rep, status))
    ms = sum(times) / len(times)
    wms = sum(wtimes) / len(wtimes)
    n, n1, n2 = ctx.sizes()
    row_blocks, ksteps = ctx.precond_layout()
    if world > 1:
        ms, wms = max_over_ranks([ms, wms], dev)
    # end to end through ff_subspace_host on pinned host buffers
    Xp, vp, ap = (torch.from_numpy(t).pin_memory() for t in (c.X, c.v, c.a))
    e2e, h2d, d2h = [], 0, 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, h2d, d2h, _ = binding.subspace_from_host(Xp, vp, ap, c.E, c.nu, 32, args.prec,
                                                          opts, local, ctx)
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    # the consumer of the modes: skinning weight fields at every particle and a
    # linear blend skinning of them (Sec. 3.2, Eq. 1)
    step()
    Zs = (0.01 * torch.randn((32, 3, 4), generator=torch.Generator().manual_seed(5))).to(
        dev, ctx.dtype)
    sk_w, sk_l = [], []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Wsk = ctx.skinning_weights(X, modes.t())
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.lbs(X, Wsk, Zs)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if i >= args.warmup:
            sk_w.append(t1 - t0)
            sk_l.append(t2 - t1)
    net.close()
    return {"ms": ms, "wms": wms, "reps": reps, "wreps": wreps, "prof": prof, "nprof": nprof,
            "pre": (pre_cnt, pre_tot), "launches": launches, "clocks": clk.summary(),
            "sizes": (n, n1, n2), "layout": (row_blocks, ksteps),
            "e2e_s": sum(e2e) / len(e2e), "h2d": h2d, "d2h": d2h,
            "sk": (1000 * sum(sk_w) / len(sk_w), 1000 * sum(sk_l) / len(sk_l))}


def torus_line(args, r, peaks):
    n, n1, n2 = r["sizes"]
    row_blocks, ksteps = r["layout"]
    cnt, tot = r["pre"]
    m = ((31 + 8 + 3) // 4) * 4
    # Chebyshev preconditioner step on the 40-column block, BF16 directions.
    # Tensor-core form: per 16-column k-step a 512 B BF16 tile and 16 int32
    # union columns, per 16-row block an int32 offset, per row the rounded row
    # sum and the diagonal (FP32); read d_in (2 B), write d_out (2 B), read and
    # write res and x (FP32): 20 B per block element.  (Sparse CUDA-core form
    # when the tiles are not built: H values and columns, row pointers, diagonal.)
    if ksteps:
        kern = "k_cheb_step_tc"
        desc = "k_cheb_step_tc (Chebyshev preconditioner step, BF16 tiles on tensor cores)"
        pre_bytes = ksteps * (512 + 64) + (row_blocks + 1) * 4 + n * 8 + 20 * n * m
    else:
        kern = "k_cheb_step_b16"
        desc = "k_cheb_step_b16 (Chebyshev preconditioner step, BF16 directions)"
        pre_bytes = n2 * 8 + (n + 1) * 8 + n * 4 + 20 * n * m
    roof = _roofline("hbm", desc, pre_bytes, "algorithmic_bytes_per_launch",
                     tot / max(cnt, 1), cnt, peaks, traffic=_traffic("precond", kern))
    scnt, stot = r["prof"]["spmm"]
    spmm_ms = stot / max(scnt, 1)
    rep, status = r["reps"][-1]
    wrep, wstatus = r["wreps"][-1]
    return {
        "workload": TORUS_WORKLOAD, "value": round(r["ms"] / 1000.0, 5), "unit": "s",
        "ms_per_step": round(r["ms"], 3), "config": torus_config(args),
        "sizes": {"n": n, "pairs": n1, "matrix_entries": n2},
        "roofline": roof,
        "spmm": {"avg_launch_ms": round(spmm_ms, 5), "launches": scnt,
                 "note": "fused (H, M) block products of both phases (FP32 values and "
                         "FP32 blocks, then double-float), mean over launches"},
        "stage_ms_per_step": {kk: round(vv[1] / r["nprof"], 3) for kk, vv in r["prof"].items()
                              if vv[0]},
        "warm": {"value": round(r["wms"] / 1000.0, 5), "unit": "s",
                 "plain_over_warm": round(r["ms"] / r["wms"], 4),
                 "iterations": wrep["iterations"], "fp32_iterations": wrep["fp32_iterations"],
                 "status": wstatus, "max_residual": wrep["max_residual"],
                 "network": "paper_2605_29318_gb300/weights/warmstart_k32.f32"},
        "solver": {"iterations": rep["iterations"], "fp32_iterations": rep["fp32_iterations"],
                   "status": status, "max_residual": rep["max_residual"],
                   "precond_spmv_calls": rep["precond_spmv_calls"]},
        "e2e": {"value": round(r["e2e_s"], 5), "unit": "s", "h2d_bytes_per_step": int(r["h2d"]),
                "d2h_bytes_per_step": int(r["d2h"]), "call": "ff_subspace_host"},
        "skinning": {"points": n, "modes": 32, "weights_ms": round(r["sk"][0], 3),
                     "lbs_ms": round(r["sk"][1], 4),
                     "weights_points_per_s": round(n / (r["sk"][0] * 1e-3))},
        "gpu_launches": int(r["launches"]), "clocks": r["clocks"],
    }


def max_over_ranks(values, device):
    """The largest of each value over all ranks of the process group (the step
    time of a replica run is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_twoset_torus(args, ctx, dev, local):
    import torch

    from paper_2605_29318_gb300 import binding, synth
    Xh, vh = synth.torus_grid(0.02)
    K, k = 1000, 32
    X = torch.from_numpy(Xh).to(dev)
    v = torch.from_numpy(vh).to(dev)
    opts = _opts(args, "twoset-torus")
    modes = torch.empty((k, K), dtype=ctx.dtype, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step():
        ctx.rkpm_build_twoset(X, v, K, 3.0, 0)
        ctx.assemble_hessian(None, None, 1e6, 0.4)
        return ctx.eigenmodes(k, opts, modes_out=modes, check=False)

    clk = Clocks(local).__enter__()
    for _ in range(args.warmup):
        _timed(step, st, flush)
    launches0 = binding.launch_count()
    times = []
    with clk:
        for _ in range(args.steps):
            t, (_, _, rep, status) = _timed(step, st, flush)
            times.append(t)
    launches = binding.launch_count() - launches0
    ctx.profile(True)
    for _ in range(args.steps):
        _timed(step, st, flush)
    prof = ctx.profile_read()
    ctx.profile(False)
    Xp, vp = torch.from_numpy(Xh).pin_memory(), torch.from_numpy(vh).pin_memory()
    host_modes = torch.empty((k, K), dtype=ctx.dtype).pin_memory()
    e2e, h2d, d2h = [], 0, 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, _, _, h2d, d2h, _ = binding.subspace_twoset_from_host(
            Xp, vp, 1e6, 0.4, K, k, 3.0, 0, args.prec, opts, local, ctx, host_modes)
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    ms = sum(times) / len(times)
    n, n1, n2 = ctx.sizes()
    line = {
        "metric": METRIC, "value": round(ms / 1000.0, 5), "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype_name(args), "data": "synthetic", "config": twoset_torus_config(args),
        "sizes": {"K": n, "pairs": n1, "matrix_entries": n2},
        "stage_ms_per_step": {kk: round(vv[1] / args.steps, 3) for kk, vv in prof.items()
                              if vv[0]},
        "solver": {"iterations": rep["iterations"], "status": status,
                   "max_residual": rep["max_residual"]},
        "e2e": {"value": round(sum(e2e) / len(e2e), 5), "unit": "s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "call": "ff_subspace_twoset_host"},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        dt = oracle_twoset_torus_step()
        line["cpu_baseline"] = {"value": round(dt, 3), "unit": "s",
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                "sample": "FP64 two-set oracle on the whole workload"}
    return line


BATCH_OBJECTS = 32
BATCH_WORKLOAD = ("batch of 32 objects (cube / torus / ellipsoid unions, seed 4, random scale "
                  "and rotation), particle counts log-uniform 2,000-200,000, k uniform 16-48, "
                  "cubic B-spline support 2.0x spacing floored at 1.5x the 8-nearest "
                  "distance, E=1e6 nu=0.4; one eigenmodes_batched call per step")


def batch_config(args):
    return {"workload": BATCH_WORKLOAD, "precision": args.prec, "tol": args.tol,
            "objects": BATCH_OBJECTS, "l2": L2_NOTE, "parallelism": "single GPU"}


def run_batch(args, dev, local):
    """Config 4 in miniature: one eigenmodes_batched call on 32 objects per
    step (a pool of host threads, one context and stream each, on one GPU);
    seconds per batch, objects/s and particles/s."""
    import torch

    from paper_2605_29318_gb300 import binding, synth
    clouds = synth.batch(BATCH_OBJECTS, seed=4)
    objs = [{"X": torch.from_numpy(c.X).to(dev), "v": torch.from_numpy(c.v).to(dev),
             "a": torch.from_numpy(c.a).to(dev), "E0": c.E, "nu0": c.nu, "k": c.k}
            for c in clouds]
    opts = _opts(args, "batch")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step():
        return binding.eigenmodes_batched(objs, args.prec, opts, device=local)

    clk = Clocks(local).__enter__()
    for _ in range(args.warmup):
        _timed(step, st, flush)
    launches0 = binding.launch_count()
    times = []
    with clk:
        for _ in range(args.steps):
            t, (status, res) = _timed(step, st, flush)
            times.append(t)
    launches = binding.launch_count() - launches0
    ms = sum(times) / len(times)
    npart = sum(c.n for c in clouds)
    return {
        "metric": METRIC, "value": round(ms / 1000.0, 5), "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype_name(args), "data": "synthetic", "config": batch_config(args),
        "batch": {"objects": len(clouds), "particles": int(npart),
                  "objects_per_s": round(len(clouds) / (ms * 1e-3), 2),
                  "particles_per_s": round(npart / (ms * 1e-3)),
                  "status": int(status),
                  "max_residual": max(r[2]["max_residual"] for r in res),
                  "iterations_max": max(r[2]["iterations"] for r in res)},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2605_29318_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    ctx = binding.Context(local, args.prec)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(local)
    # FP32 pipe peak from the unit counts: SMs x 128 FP32 lanes x 2 (FMA) x max clock
    peaks["fp32_tflops"] = round(props.multi_processor_count * 128 * 2 * peaks["sm_max_mhz"]
                                 * 1e-6, 2)
    if args.workload == "batch":
        line = run_batch(args, dev, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        ctx.close()
        return
    if args.workload == "twoset-torus":
        line = run_twoset_torus(args, ctx, dev, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        ctx.close()
        return
    if args.workload == "torus":
        r = run_torus(args, ctx, dev, local, rank, world)
        if rank == 0:
            t = torus_line(args, r, peaks)
            line = {"metric": METRIC, "value": t["value"], "unit": "s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": t["ms_per_step"],
                    "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                    "dtype": _dtype_name(args), "data": "synthetic"}
            t["config"]["parallelism"] = "replicas" if world > 1 else "single GPU"
            line.update({kk: vv for kk, vv in t.items() if kk not in ("value", "unit",
                                                                      "ms_per_step", "workload")})
            if not args.no_cpu_baseline and world == 1:
                line["cpu_baseline"] = {
                    "value": round(oracle_torus_step(), 3), "unit": "s",
                    "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                    "sample": "FP64 oracle on the same torus with 10,000 particles instead of "
                              "50,000 (not scaled)"}
            print(json.dumps(line), flush=True)
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return
    # default: the splat workload, the torus beside it
    r = run_splat(args, ctx, dev, local)
    ms = r["ms"]
    if world > 1:
        ms = max_over_ranks([ms], dev)[0]
        r["ms"] = ms
    r["pair_products"] = ctx.pair_products()
    tor = None
    if not args.no_torus:
        tctx = binding.Context(local, args.prec)
        tor = run_torus(args, tctx, dev, local, rank, world)
        tctx.close()
    if rank == 0:
        line = splat_line(args, r, peaks)
        line["n_gpus"] = world
        if world > 1:
            line["config"]["parallelism"] = "replicas"
        if tor is not None:
            line["torus50k"] = torus_line(args, tor, peaks)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline_splat()
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only), on
    the same workload and config as our arm; each step a bounded sample scaled
    to the whole workload (the splat), the whole workload (the two-set torus),
    or a 10,000-particle sample of the nodal torus."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    if args.workload == "splat":
        o = OracleSplat()
        one, config, sample = (lambda: o.step()[0]), splat_config(args), o.describe()
    elif args.workload == "twoset-torus":
        one, config = oracle_twoset_torus_step, twoset_torus_config(args)
        sample = "FP64 two-set oracle on the whole workload"
    elif args.workload == "batch":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the batch workload has no oracle arm (its objects are checked "
                          "one by one against the single-object calls)"}), flush=True)
        return
    else:
        one, config = oracle_torus_step, torus_config(args)
        sample = "FP64 oracle on the same torus with 10,000 particles instead of 50,000"
    for _ in range(args.warmup):
        one()
    times = [one() for _ in range(args.steps)]
    v = sum(times) / len(times)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * v, 2), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 4), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="splat",
                    choices=["splat", "torus", "twoset-torus", "batch"],
                    help="the splat-like cloud (default), the nodal torus, the two-set torus, "
                         "or a 32-object batch")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--cheb", type=int, default=None,
                    help="FP32 preconditioner degree (default: 32 for the splat, 16 otherwise)")
    ap.add_argument("--cheb-fp64", type=int, default=None,
                    help="double-float phase preconditioner degree (default 48)")
    ap.add_argument("--fp32-phase", type=int, default=1, choices=[0, 1],
                    help="FP64 contexts: iterate in FP32 first, then finish in double-float")
    ap.add_argument("--max-iter", type=int, default=500)
    ap.add_argument("--fp32-tol", type=float, default=None,
                    help="residual at which the FP32 phase hands over (default: 3e-5 for the "
                         "splat, 1e-4 otherwise)")
    ap.add_argument("--precond-tc", type=int, default=1, choices=[0, 1],
                    help="preconditioner steps on tensor cores (BF16 tiles) or on CUDA cores")
    ap.add_argument("--precond-compact", type=int, default=0, choices=[0, 1],
                    help="preconditioner steps on the unconverged columns only, packed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--build-prec", default=None, choices=["fp64", "fp32"],
                    help="splat: shape functions and assembly sums in double-float (fp64) or "
                         "FP32 (the matrices stored in FP64 either way; default fp32)")
    ap.add_argument("--no-torus", action="store_true",
                    help="splat workload: leave out the nodal torus beside it")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
