"""Fixed cases of the hot path for a profiler (ncu) to capture.

    python -m paper_2605_29318_gb300.profile_case splat [steps]
        the 1,000,000-point splat through the two-set construction (K = 1,000,
        k = 64, FP64 context, default options): rkpm_build_twoset +
        assemble_hessian + eigenmodes, `steps` times (2 by default)
    python -m paper_2605_29318_gb300.profile_case torus [steps]
        the 50,000-particle solid torus, nodal (k = 32, FP64 context)
    python -m paper_2605_29318_gb300.profile_case twoset [steps]
        the two-set build and assembly alone on the solid torus's inside grid at
        h = 0.012 (228,357 points, K = 1,000): a case of the splat's kernels
        (whole-GPU farthest-point sampling, Gaussian shape functions, dense-tile
        assembly) that holds about 1 GB on the device
    python -m paper_2605_29318_gb300.profile_case twoset32 [steps]
        the same with FP32 build precision (the splat benchmark's setting)
    python -m paper_2605_29318_gb300.profile_case splat32 [steps]
        the splat step as the benchmark runs it (FP32 build precision, FP32
        preconditioner degree 32, hand-over from the FP32 phase at 3e-5)

Each step is synchronised; the script prints the solver status and iteration
count.  It only drives the library (nothing is timed here).
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv):
    import numpy as np
    import torch

    from paper_2605_29318_gb300 import binding, synth
    case = argv[1] if len(argv) > 1 else "splat"
    steps = int(argv[2]) if len(argv) > 2 else 2
    dev = "cuda:0"
    ctx = binding.Context(0, "fp64")
    opts = binding.default_opts()
    if case in ("splat32", "twoset32"):
        ctx.set_build_precision("fp32")
    if case == "splat32":
        opts = binding.default_opts(cheb_degree=32, cheb_degree_fp64=48, fp32_tol=3e-5)
    if case in ("splat", "splat32"):
        c = synth.gaussian_mixture(1_000_000)
        X, v = torch.from_numpy(c.X).to(dev), torch.from_numpy(c.v).to(dev)
        E = torch.from_numpy(np.ascontiguousarray(c.E, np.float32)).to(dev)
        modes = torch.empty((64, 1000), dtype=torch.float64, device=dev)
        for _ in range(steps):
            ctx.rkpm_build_twoset(X, v, 1000, 3.0, 0)
            ctx.assemble_hessian(E, None, 1.0, float(c.nu))
            _, _, rep, st = ctx.eigenmodes(64, opts, modes_out=modes, check=False)
            torch.cuda.synchronize()
            print("splat step", st, rep["iterations"], flush=True)
    elif case == "torus":
        c = synth.torus(50000, seed=2)
        X, v, a = (torch.from_numpy(t).to(dev) for t in (c.X, c.v, c.a))
        for _ in range(steps):
            ctx.rkpm_build(X, v, a)
            ctx.assemble_hessian(None, None, c.E, c.nu)
            _, _, rep, st = ctx.eigenmodes(32, opts, check=False)
            torch.cuda.synchronize()
            print("torus step", st, rep["iterations"], flush=True)
    elif case in ("twoset", "twoset32"):
        Xq, vq = synth.torus_grid(0.012)
        X, v = torch.from_numpy(Xq).to(dev), torch.from_numpy(vq).to(dev)
        for _ in range(steps):
            ctx.rkpm_build_twoset(X, v, 1000, 3.0, 0)
            ctx.assemble_hessian(None, None, 1e6, 0.4)
            torch.cuda.synchronize()
            print("twoset build", ctx.sizes(), flush=True)
    else:
        raise SystemExit(f"unknown case {case!r} (splat, splat32, torus, twoset, twoset32)")
    ctx.close()


if __name__ == "__main__":
    main(sys.argv)
