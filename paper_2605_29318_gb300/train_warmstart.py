"""Train the warm-start network on procedural shapes and evaluate it.

    python -m paper_2605_29318_gb300.train_warmstart [--train 96] [--heldout 16]
        [--nmin 8000] [--nmax 30000] [--epochs 60] [--out DIR]
    python -m paper_2605_29318_gb300.train_warmstart --eval-only --heldout 100 \
        --nmin 20000 --nmax 100000

Labels are the 31 lowest non-constant modes (k = 32) of each training shape,
computed by this library's own plain eigensolver path (FP32 context, random
start, relative residual 1e-4).  Training runs the library's forward, loss,
backward and Adam kernels (ff_net_train_step) one shape per step with a cosine
learning-rate schedule.  The held-out evaluation solves each held-out shape to
relative residual 1e-6 in an FP64 context twice, from the random start and
from the network's start block, and records iterations and wall time.

Writes DIR/warmstart_k32.f32 (the flat FP32 parameters) and
DIR/warmstart_k32.json (corpus, schedule, losses, held-out results).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import binding, synth

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "warmstart_k32.f32")


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    theta = np.fromfile(path, dtype=np.float32)
    if theta.size != 170784:
        raise ValueError(f"{path}: expected 170784 parameters, found {theta.size}")
    return theta


def _cloud_tensors(c):
    import torch
    X, v, a = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (c.X, c.v, c.a))
    return X, v, a


def label_shape(c, k=32, tol=1e-4):
    """(features, volumes, modes (k-1, n)) on the device for one cloud."""
    ctx = binding.Context(0, "fp32")
    X, v, a = _cloud_tensors(c)
    ctx.rkpm_build(X, v, a)
    ctx.assemble_hessian(None, None, c.E, c.nu)
    o = binding.default_opts(tol=tol, max_iter=300)
    ev, modes, rep, st = ctx.eigenmodes(k, o, check=False)
    feat = ctx.warmstart_features()
    lab = modes.t()[1:].contiguous()          # (k - 1, n): column-major n x (k - 1)
    ctx.close()
    return feat, v, lab, rep


def solve_time(c, net=None, k=32, tol=1e-6):
    """Wall time (s) and iterations of rkpm_build .. eigenmodes in FP64 (features
    and inference included for the warm start)."""
    import torch
    X, v, a = _cloud_tensors(c)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = binding.Context(0, "fp64")
    ctx.rkpm_build(X, v, a)
    ctx.assemble_hessian(None, None, c.E, c.nu)
    o = binding.default_opts(tol=tol)
    X0 = ctx.warmstart_block(net, k, o) if net is not None else None
    ev, modes, rep, st = ctx.eigenmodes(k, o, X0=X0, check=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.close()
    return dt, rep, st


def evaluate(n_heldout=100, nmin=20000, nmax=100000, path=None, k=32, tol=1e-6, repeats=2):
    """The trained network against the random start on held-out shapes (seeds
    20000 + i, particle counts log-uniform in [nmin, nmax]): per shape one
    context, a warm-up solve, then the best of `repeats` device-timed steps
    (rkpm_build + assemble_hessian [+ features and inference] + eigenmodes to
    relative residual tol, FP64 context) from each start.  Returns the
    per-shape records and the distribution of iterations, times and their
    ratios."""
    import torch
    net = binding.Net(0)
    net.set_params(load_weights() if path is None else load_weights(path))
    recs = []
    st = torch.cuda.current_stream()
    for i in range(n_heldout):
        c = synth.warmstart_shape(20000 + i, nmin, nmax, k)
        X, v, a = _cloud_tensors(c)
        ctx = binding.Context(0, "fp64")
        o = binding.default_opts(tol=tol)

        def step(warm):
            ctx.rkpm_build(X, v, a)
            ctx.assemble_hessian(None, None, c.E, c.nu)
            X0 = ctx.warmstart_block(net, k, o) if warm else None
            return ctx.eigenmodes(k, o, X0=X0, check=False)

        out = {}
        for warm in (False, True):
            step(warm)
            best, rep, status = math.inf, None, None
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                _, _, rep, status = step(warm)
                e1.record(st)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1000.0)
            out[warm] = (best, rep, status)
        recs.append(dict(name=c.name, n=c.n, plain_s=out[False][0], warm_s=out[True][0],
                         plain_iters=out[False][1]["iterations"],
                         warm_iters=out[True][1]["iterations"],
                         plain_status=out[False][2], warm_status=out[True][2]))
        print(json.dumps(recs[-1]), flush=True)
        ctx.close()
    net.close()
    ratio = np.array([r["plain_s"] / r["warm_s"] for r in recs])
    dit = np.array([r["plain_iters"] - r["warm_iters"] for r in recs])
    q = [10, 50, 90]
    summary = dict(
        shapes=len(recs), nmin=nmin, nmax=nmax, tol=tol,
        plain_over_warm_time=dict(zip(["p10", "p50", "p90"], np.percentile(ratio, q).tolist()),
                                  mean=float(ratio.mean())),
        iterations_saved=dict(zip(["p10", "p50", "p90"], np.percentile(dit, q).tolist()),
                              mean=float(dit.mean())),
        plain_s_mean=float(np.mean([r["plain_s"] for r in recs])),
        warm_s_mean=float(np.mean([r["warm_s"] for r in recs])),
        all_converged=bool(all(r["plain_status"] == 0 and r["warm_status"] == 0 for r in recs)))
    return recs, summary


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=96)
    ap.add_argument("--heldout", type=int, default=16)
    ap.add_argument("--nmin", type=int, default=8000)
    ap.add_argument("--nmax", type=int, default=30000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=os.path.dirname(WEIGHTS))
    ap.add_argument("--eval-only", action="store_true",
                    help="evaluate the stored network on --heldout shapes of --nmin..--nmax "
                         "particles and write DIR/warmstart_k32_eval.json")
    args = ap.parse_args(argv)
    import torch
    if args.eval_only:
        recs, summary = evaluate(args.heldout, args.nmin, args.nmax)
        with open(os.path.join(args.out, "warmstart_k32_eval.json"), "w") as fh:
            json.dump(dict(summary=summary, shapes=recs), fh, indent=1)
        print(json.dumps(summary), flush=True)
        return

    t0 = time.perf_counter()
    data = []
    for i in range(args.train):
        c = synth.warmstart_shape(10000 + i, args.nmin, args.nmax)
        feat, v, lab, rep = label_shape(c)
        data.append((feat, v, lab))
    t_label = time.perf_counter() - t0

    net = binding.Net(0, seed=args.seed)
    rng = np.random.default_rng(args.seed)
    steps = args.epochs * len(data)
    hist = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(args.epochs):
        losses = []
        for j in rng.permutation(len(data)):
            lr = args.lr * (0.01 + 0.99 * 0.5 * (1 + math.cos(math.pi * step / steps)))
            losses.append(net.train_step(*data[j], lr))
            step += 1
        hist.append(float(np.mean(losses)))
        print(f"epoch {ep}: mean loss {hist[-1]:.4f}", flush=True)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    os.makedirs(args.out, exist_ok=True)
    theta = net.get_params()
    theta.tofile(os.path.join(args.out, "warmstart_k32.f32"))

    # held-out: loss against the plain path's modes, then solve times
    held = []
    for i in range(args.heldout):
        c = synth.warmstart_shape(20000 + i, args.nmin, args.nmax)
        feat, v, lab, _ = label_shape(c)
        loss = net.loss_grad(feat, v, lab)[0]
        tp, rp, sp = solve_time(c)
        tw, rw, sw = solve_time(c, net)
        held.append(dict(name=c.name, n=c.n, loss=loss, plain_s=tp, warm_s=tw,
                         plain_iters=rp["iterations"], warm_iters=rw["iterations"],
                         plain_status=sp, warm_status=sw))
        print(json.dumps(held[-1]), flush=True)
    summary = dict(
        corpus=dict(train_seeds=[10000, 10000 + args.train - 1],
                    heldout_seeds=[20000, 20000 + args.heldout - 1],
                    nmin=args.nmin, nmax=args.nmax, k=32, label_tol=1e-4),
        schedule=dict(epochs=args.epochs, lr=args.lr, seed=args.seed, steps=steps,
                      optimiser="Adam(0.9, 0.999, 1e-8), cosine to 1% of lr"),
        seconds=dict(labels=t_label, training=t_train),
        epoch_loss=hist,
        heldout=held,
        heldout_mean=dict(
            loss=float(np.mean([h["loss"] for h in held])) if held else None,
            plain_s=float(np.mean([h["plain_s"] for h in held])) if held else None,
            warm_s=float(np.mean([h["warm_s"] for h in held])) if held else None,
            plain_iters=float(np.mean([h["plain_iters"] for h in held])) if held else None,
            warm_iters=float(np.mean([h["warm_iters"] for h in held])) if held else None),
    )
    with open(os.path.join(args.out, "warmstart_k32.json"), "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps(summary["heldout_mean"]), flush=True)
    net.close()


if __name__ == "__main__":
    main()
