"""Benchmark of the subspace-construction hot path on GB300.

One step = rkpm_build + assemble_hessian + eigenmodes on the seeded solid torus
(R = 0.5, r = 0.2, 50,000 particles, support 2.0x spacing, E = 1e6, nu = 0.4,
k = 32 modes with the constant one) with the inputs already resident in HBM.
The metric is the time to k modes at relative residual 1e-6: `value` is the
plain path (seeded random start block); `warm` times the same step started
from the trained warm-start network (features and inference included).  L2 is
flushed (a 256 MB write) before every timed step; each step is timed with CUDA
events on the library's stream.  The line also reports the end-to-end time
from host arrays (`e2e`), the roofline of the preconditioner step, the stage
split, and the evaluation of the modes' skinning weight fields at every
particle with a linear blend skinning of them (`skinning`).  Prints one JSON
line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec fp64|fp32] [--tol T] [--cheb D] [--cheb-fp64 D]
                  [--fp32-phase 0|1] [--fp32-tol T] [--precond-tc 0|1]
                  [--precond-compact 0|1] [--workload nodal|twoset]

`--workload twoset` times the paper's own two-set construction instead: the
same torus as 49,584 grid quadrature points (h = 0.02), K = 1,000
farthest-point centres with Gaussian kernels cut at 3 r_k, the same material
and k; one step = rkpm_build_twoset + assemble_hessian + eigenmodes.

With N > 1 (torchrun, one process per GPU) every rank solves its own object
(replicas; the path has no cross-GPU exchange) and the reported time is the
maximum over ranks.  `--impl reference` times the FP64 CPU oracle on the host
cores on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-k-modes at rel. residual 1e-6 (s), warm vs plain; SpMM HBM GB/s"
WORKLOAD = ("solid torus R=0.5 r=0.2, 50,000 particles rejection-sampled (seed 2), "
            "cubic B-spline support 2.0x spacing, Neo-Hookean E=1e6 nu=0.4, "
            "k=32 lowest modes incl. the constant mode")
SAMPLE_N = 10000  # bounded oracle sample (same torus, 10,000 particles)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


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
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

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


def cpu_oracle_step(n=SAMPLE_N, k=32):
    """The FP64 oracle's whole path on the bounded sample: brute-force
    neighbours, shape functions, sparse H_w and M, shift-invert eigensolve."""
    from oracle import assembly, eigen, rkpm
    from paper_2605_29318_gb300 import synth
    c = synth.torus(n, seed=2)
    t0 = time.perf_counter()
    ptr, idx = rkpm.neighbours(c.X, c.a, chunk=64)
    phi, dphi, _ = rkpm.shape_functions(c.X, c.a, ptr, idx)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam, C = eigen.eigsh_sparse(H, M, k)
    dt = time.perf_counter() - t0
    return dt, float(eigen.residuals(H, M, lam, C)[1:].max())


def cpu_baseline_json():
    dt, res = cpu_oracle_step()
    return {"value": round(dt, 3), "unit": "s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle",
            "sample": (f"FP64 oracle (brute-force neighbours, shape functions, scipy sparse "
                       f"H_w/M, shift-invert eigsh k=32) on the same torus with {SAMPLE_N:,} "
                       f"particles instead of 50,000; not scaled"),
            "max_residual": res}


TWOSET_WORKLOAD = ("solid torus R=0.5 r=0.2 as 49,584 inside-grid quadrature points "
                   "(h=0.02), K=1,000 farthest-point centres, Gaussian kernels with "
                   "r_k = 2nd-nearest-centre distance cut at 3 r_k, Neo-Hookean E=1e6 "
                   "nu=0.4, k=32 lowest modes incl. the constant mode")
def cpu_twoset_step(h=0.02, K=1000, k=32):
    """The FP64 oracle's two-set path on the whole workload (a few seconds):
    farthest-point centres, radii, Gaussian shape functions, dense H_w and M,
    dense eigensolve."""
    from oracle import eigen, twoset
    from paper_2605_29318_gb300 import synth
    X, v = synth.torus_grid(h)
    t0 = time.perf_counter()
    _, _, H, M = twoset.build(X, v, K, 1e6, 0.4, trunc=3.0)
    lam, C = eigen.eigh_dense(H, M, k)
    dt = time.perf_counter() - t0
    return dt, float(eigen.residuals(H, M, lam, C)[1:].max()), X.shape[0]


def run_twoset(args):
    """One GPU, the two-set workload: device-timed steps (L2 flushed), the
    stage split, and the end-to-end step from host arrays."""
    import numpy as np
    import torch

    from paper_2605_29318_gb300 import binding, synth
    torch.cuda.set_device(0)
    dev = "cuda:0"
    Xh, vh = synth.torus_grid(0.02)
    K, k = 1000, 32
    X = torch.from_numpy(Xh).to(dev)
    v = torch.from_numpy(vh).to(dev)
    ctx = binding.Context(0, args.prec)
    opts = binding.default_opts(tol=args.tol, cheb_degree=args.cheb, max_iter=args.max_iter,
                                fp32_phase=args.fp32_phase, cheb_degree_fp64=args.cheb_fp64,
                                precond_tc=args.precond_tc, fp32_tol=args.fp32_tol,
                                precond_compact=args.precond_compact)
    modes = torch.empty((k, K), dtype=ctx.dtype, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step(Xd, vd):
        ctx.rkpm_build_twoset(Xd, vd, K, 3.0, 0)
        ctx.assemble_hessian(None, None, 1e6, 0.4)
        return ctx.eigenmodes(k, opts, modes_out=modes, check=False)

    for _ in range(args.warmup):
        flush.zero_()
        step(X, v)
    torch.cuda.synchronize()
    ctx.profile(True)
    launches0 = binding.launch_count()
    times = []
    with Clocks(0) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            _, _, rep, status = step(X, v)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    launches = binding.launch_count() - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = sum(times) / len(times)
    # end to end: pinned host inputs copied in, the modes read back, per step
    Xp, vp = torch.from_numpy(Xh).pin_memory(), torch.from_numpy(vh).pin_memory()
    host_modes = torch.empty((k, K), dtype=ctx.dtype).pin_memory()
    e2e = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd, vd = Xp.to(dev, non_blocking=True), vp.to(dev, non_blocking=True)
        step(Xd, vd)
        host_modes.copy_(modes)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    e2e_s = sum(e2e) / len(e2e)
    n, n1, n2 = ctx.sizes()
    line = {
        "metric": METRIC, "value": round(ms / 1000.0, 5), "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": (("f32+bf16, then f32x2 double-float" if args.fp32_phase
                   else "f64") if args.prec == "fp64" else "f32+bf16"),
        "data": "synthetic",
        "config": {"workload": TWOSET_WORKLOAD, "precision": args.prec, "tol": args.tol,
                   "quadrature_points": int(Xh.shape[0]), "K": n, "n1": n1, "n2": n2,
                   "l2": "flushed by a 256 MB write before every timed step",
                   "parallelism": "single GPU"},
        "stage_ms_per_step": {kk: round(vv[1] / args.steps, 3) for kk, vv in prof.items()},
        "solver": {"iterations": rep["iterations"], "status": status,
                   "max_residual": rep["max_residual"]},
        "e2e": {"value": round(e2e_s, 5), "unit": "s",
                "h2d_bytes_per_step": int(Xh.nbytes + vh.nbytes),
                "d2h_bytes_per_step": int(host_modes.numel() * host_modes.element_size())},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        dt, res, npts = cpu_twoset_step()
        line["cpu_baseline"] = {
            "value": round(dt, 3), "unit": "s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "max_residual": res,
            "sample": (f"FP64 two-set oracle (farthest-point centres, radii, Gaussian shape "
                       f"functions, dense H_w/M, dense eigensolve) on the whole workload "
                       f"({npts:,} points, K=1,000)")}
    print(json.dumps(line), flush=True)
    ctx.close()


def max_over_ranks(values, device):
    """The largest of each value over all ranks of the process group (the step
    time of a replica run is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    twoset = args.workload == "twoset"
    one = (lambda: cpu_twoset_step()[:2]) if twoset else cpu_oracle_step
    for _ in range(args.warmup):
        one()
    times = []
    res = None
    for _ in range(args.steps):
        dt, res = one()
        times.append(dt)
    v = sum(times) / len(times)
    cores = len(os.sched_getaffinity(0))
    if twoset:
        workload, sample = TWOSET_WORKLOAD, "the whole workload (49,584 points, K=1,000)"
    else:
        workload = WORKLOAD
        sample = f"oracle on the same torus with {SAMPLE_N:,} particles"
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * v, 2), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "sample": sample},
            "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": cores,
                             "kind": "oracle", "sample": sample + ", k=32"},
            "e2e": {"value": round(v, 4), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "max_residual": res}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2605_29318_gb300 import binding, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    c = synth.torus(50000, seed=2 + 1000 * rank)
    X = torch.from_numpy(c.X).to(dev)
    v = torch.from_numpy(c.v).to(dev)
    a = torch.from_numpy(c.a).to(dev)
    ctx = binding.Context(local, args.prec)
    opts = binding.default_opts(tol=args.tol, cheb_degree=args.cheb, max_iter=args.max_iter,
                                fp32_phase=args.fp32_phase, cheb_degree_fp64=args.cheb_fp64,
                                precond_tc=args.precond_tc, fp32_tol=args.fp32_tol,
                                precond_compact=args.precond_compact)
    from paper_2605_29318_gb300 import train_warmstart
    net = binding.Net(local)
    net.set_params(train_warmstart.load_weights())
    modes = torch.empty((32, c.n), dtype=ctx.dtype, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step(warm=False):
        ctx.rkpm_build(X, v, a)
        ctx.assemble_hessian(None, None, c.E, c.nu)
        X0 = ctx.warmstart_block(net, 32, opts) if warm else None
        ev, _, rep, status = ctx.eigenmodes(32, opts, X0=X0, modes_out=modes, check=False)
        return ev, rep, status

    def timed(warm):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        ev, rep, status = step(warm)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), rep, status

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ctx.profile(True)
    launches0 = binding.launch_count()
    times, reps = [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            t, rep, status = timed(False)
            times.append(t)
            reps.append((rep, status))
    launches = binding.launch_count() - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    # the same step from the learned warm start
    for _ in range(args.warmup):
        timed(True)
    wtimes, wreps = [], []
    for _ in range(args.steps):
        t, rep, status = timed(True)
        wtimes.append(t)
        wreps.append((rep, status))
    wms = sum(wtimes) / len(wtimes)
    n, n1, n2 = ctx.sizes()
    ms = sum(times) / len(times)
    if world > 1:
        ms, wms = max_over_ranks([ms, wms], dev)
        dist.barrier()

    # end to end through the public call on host buffers (H2D + D2H inside)
    e2e = []
    h2d = d2h = 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, h2d, d2h, _ = binding.subspace_from_host(c.X, c.v, c.a, c.E, c.nu, 32,
                                                          args.prec, opts, local, ctx)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    e2e_s = sum(e2e) / len(e2e)

    # the consumer of the modes: their skinning weight fields at every particle
    # and a linear blend skinning of them (Sec. 3.2, Eq. 1), wall time per call
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
    sk_w_ms, sk_l_ms = 1000 * sum(sk_w) / len(sk_w), 1000 * sum(sk_l) / len(sk_l)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    # dominant kernel: the Chebyshev preconditioner step (H-only block product
    # on the 40-column block, BF16 directions).  Tensor-core form: per 16-column
    # k-step a 512 B BF16 tile and 16 int32 union columns, per 16-row block an
    # int32 offset, per row the rounded row sum and the diagonal (FP32); read
    # d_in (2 B), write d_out (2 B), read and write res and x (FP32): 20 B per
    # block element.  (Sparse CUDA-core form when the tiles are not built: H
    # values and columns, row pointers, diagonal.)
    cnt, tot = prof["precond"]
    m = ((31 + 8 + 3) // 4) * 4
    row_blocks, ksteps = ctx.precond_layout()
    if ksteps:
        pre_kernel = "k_cheb_step_tc"
        pre_desc = "k_cheb_step_tc (Chebyshev preconditioner step, BF16 tiles on tensor cores)"
        pre_bytes = ksteps * (512 + 64) + (row_blocks + 1) * 4 + n * 8 + 20 * n * m
    else:
        pre_kernel = "k_cheb_step_b16"
        pre_desc = "k_cheb_step_b16 (Chebyshev preconditioner step, BF16 directions)"
        pre_bytes = n2 * 8 + (n + 1) * 8 + n * 4 + 20 * n * m
    pre_ms = tot / max(cnt, 1)
    achieved = pre_bytes / (pre_ms * 1e-3) / 1e9 if cnt else None
    tr = _traffic("precond", pre_kernel)
    # secondary: fused (H, M) block product
    scnt, stot = prof["spmm"]
    t_el = 8 if args.prec == "fp64" else 4
    spmm_bytes = n2 * (2 * t_el + 4) + (n + 1) * 8 + 3 * n * m * t_el
    spmm_gbs = spmm_bytes / (stot / max(scnt, 1) * 1e-3) / 1e9 if scnt else None
    last_rep, last_status = reps[-1]
    line = {
        "metric": METRIC, "value": round(ms / 1000.0, 5), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": (("f32+bf16, then f32x2 double-float" if args.fp32_phase
                   else "f64") if args.prec == "fp64" else "f32+bf16"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.prec, "tol": args.tol,
                   "cheb_degree": args.cheb, "cheb_degree_fp64": args.cheb_fp64,
                   "precond_tc": args.precond_tc, "fp32_tol": args.fp32_tol,
                   "precond_compact": args.precond_compact,
                   "n": n, "n1": n1, "n2": n2,
                   "l2": "flushed by a 256 MB write before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"kernel": pre_desc,
                     "bound": "hbm", "achieved": round(achieved, 1) if achieved else None,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4) if achieved else None,
                     "traffic": tr, "algorithmic_bytes_per_launch": pre_bytes,
                     "avg_launch_ms": round(pre_ms, 5), "launches": cnt},
        "skinning": {"points": n, "modes": 32, "weights_ms": round(sk_w_ms, 3),
                     "lbs_ms": round(sk_l_ms, 4),
                     "weights_points_per_s": round(n / (sk_w_ms * 1e-3))},
        "spmm": {"avg_launch_ms": round(stot / max(scnt, 1), 5), "launches": scnt,
                 "algorithmic_gbs": round(spmm_gbs, 1) if spmm_gbs else None,
                 "note": "average over both phases' launches, bytes counted at the second "
                         "phase's 8-byte elements"},
        "stage_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in prof.items()},
        "warm": {"value": round(wms / 1000.0, 5), "unit": "s",
                 "plain_over_warm": round(ms / wms, 4),
                 "iterations": wreps[-1][0]["iterations"],
                 "fp32_iterations": wreps[-1][0]["fp32_iterations"],
                 "status": wreps[-1][1], "max_residual": wreps[-1][0]["max_residual"],
                 "network": "paper_2605_29318_gb300/weights/warmstart_k32.f32"},
        "solver": {"iterations": last_rep["iterations"],
                   "fp32_iterations": last_rep["fp32_iterations"], "status": last_status,
                   "max_residual": last_rep["max_residual"],
                   "precond_spmv_calls": last_rep["precond_spmv_calls"]},
        "e2e": {"value": round(e2e_s, 5), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_json()
    print(json.dumps(line), flush=True)
    net.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--cheb", type=int, default=16)
    ap.add_argument("--cheb-fp64", type=int, default=64)
    ap.add_argument("--fp32-phase", type=int, default=1, choices=[0, 1],
                    help="FP64 contexts: iterate in FP32 first, then finish in FP64")
    ap.add_argument("--max-iter", type=int, default=500)
    ap.add_argument("--fp32-tol", type=float, default=1e-4,
                    help="residual at which the FP32 phase hands over")
    ap.add_argument("--precond-tc", type=int, default=1, choices=[0, 1],
                    help="preconditioner steps on tensor cores (BF16 tiles) or on CUDA cores")
    ap.add_argument("--precond-compact", type=int, default=0, choices=[0, 1],
                    help="preconditioner steps on the unconverged columns only, packed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="nodal", choices=["nodal", "twoset"],
                    help="the nodal torus (default) or the paper's two-set construction")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "twoset":
        run_twoset(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
