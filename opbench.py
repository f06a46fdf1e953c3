"""Operator microbenchmark: times one libgpe entry point on a synthetic field.

    python opbench.py --grid 256 256 512 --prec mixed --op apply_H --iters 20

Prints one JSON line: median CUDA-event time per call, points, and the
effective bandwidth for the given algorithmic bytes per point.  Also used as
the small, self-contained program for ncu captures of single passes.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs="+", default=[256, 256, 512])
    ap.add_argument("--L", type=float, default=8.0)
    ap.add_argument("--prec", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--op", choices=["apply_H", "apply_H_batch", "precond", "energy", "solve"], default="apply_H")
    ap.add_argument("--batch", type=int, default=64, help="fields for --op apply_H_batch (2D grid)")
    ap.add_argument("--hbatch-E", type=int, default=0, help="values per thread of the batched H kernel (8, 16)")
    ap.add_argument("--hbatch-rows", type=int, default=16, help="rows per CTA of its streaming form (16, 32)")
    ap.add_argument("--workload", default="fast256_2d", help="for --op solve")
    ap.add_argument("--max-iter", type=int, default=50, help="for --op solve")
    ap.add_argument("--switch-res", type=float, default=0.0, help="for --op solve (mixed)")
    ap.add_argument("--loop", choices=["default", "cluster", "persistent", "graph", "host"], default="default",
                    help="for --op solve: the library default, the cluster-resident complex64 phase, the "
                         "persistent kernel, the graph with a device-side loop, or a host loop")
    ap.add_argument("--autotune", action="store_true", help="for --op solve: tune the pass-kernel plans first")
    ap.add_argument("--plan", default="",
                    help="E,width applied to every axis (solve: every mode), or E,w/E,w[/E,w] per axis")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args()

    import torch

    from paper_1611_02045_gb300 import build, gpe, inputs as I
    build.build()
    dev = torch.device("cuda", 0)
    prec = gpe.GPE_FP64 if a.prec == "fp64" else gpe.GPE_MIXED
    stream = torch.cuda.current_stream()

    if a.op == "solve":
        w = I.workload(a.workload)
        ctx = gpe.Context(w["n"], w["L"], w["eta"], w["omega"], w["V"], prec=prec)
        if a.autotune:
            ctx.autotune(iters=20)
        if a.plan:
            E, wd = (int(v) for v in a.plan.split(","))
            for m in ((0, 1, 2) if prec == gpe.GPE_MIXED else (1,)):
                for ax in range(len(w["n"])):
                    ctx.set_plan(m, ax, E, wd)
        phi0 = torch.from_numpy(w["phi0"].copy()).to(dev)
        phi = torch.empty_like(phi0)
        opts = gpe.solve_opts_default()
        opts.max_iter = a.max_iter
        opts.switch_res = a.switch_res
        if a.loop != "default":
            opts.use_graph = {"cluster": 3, "persistent": 2, "graph": 1, "host": 0}[a.loop]
        times = []
        for i in range(a.warmup + a.iters):
            phi.copy_(phi0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = ctx.pcg_solve(phi, opts)
            e1.record(stream)
            e1.synchronize()
            if i >= a.warmup:
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        print(json.dumps({"op": "solve", "workload": a.workload, "prec": a.prec, "max_iter": a.max_iter,
                          "loop": a.loop, "loop_kind": rep["loop_kind"], "iters": rep["iters"], "iters_lo": rep["iters_lo"], "ms": ms,
                          "ms_per_iter": ms / max(rep["iters"], 1)}))
        return

    n = tuple(a.grid)
    N = int(np.prod(n))
    L = (a.L,) * len(n)
    V = torch.zeros(N, dtype=torch.float64, device=dev)
    ctx = gpe.Context(n, L, 100.0, 0.5, V, prec=prec)
    del V
    if a.hbatch_E:
        ctx.set_plan(3, 0, a.hbatch_E, a.hbatch_rows)
    if a.plan:
        per = a.plan.split("/")
        for ax in range(len(n)):
            E, wd = (int(v) for v in per[ax if len(per) > 1 else 0].split(","))
            ctx.set_plan(1 if prec == gpe.GPE_FP64 else 0, ax, E, wd)
    dt = torch.complex128 if a.prec == "fp64" else torch.complex64
    g = torch.Generator(device=dev).manual_seed(1)
    nf = a.batch if a.op == "apply_H_batch" else 1
    phi = torch.randn(N * nf, dtype=dt, device=dev, generator=g)
    out = torch.empty_like(phi)
    cb = 16 if a.prec == "fp64" else 8
    vb = 8 if a.prec == "fp64" else 4
    if a.op == "apply_H":
        call = lambda: ctx.apply_H(phi, phi, out)  # noqa: E731
        bytes_pt = 2 * cb + vb
    elif a.op == "apply_H_batch":
        call = lambda: ctx.apply_H_batch(nf, phi, phi, out)  # noqa: E731
        bytes_pt = 2 * cb + vb / nf  # V is read once for the batch
    elif a.op == "precond":
        call = lambda: ctx.precond(phi, phi, 1.5, out)  # noqa: E731
        bytes_pt = 3 * cb + vb
    else:
        call = lambda: ctx.energy(phi)  # noqa: E731
        bytes_pt = cb + vb
    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    plan = [list(ctx.get_plan(1 if prec == gpe.GPE_FP64 else 0, ax)) for ax in range(len(n))]
    print(json.dumps({"op": a.op, "grid": list(n), "fields": nf, "prec": a.prec, "plan": plan, "points": N * nf, "ms": ms,
                      "algorithmic_bytes_per_point": bytes_pt,
                      "effective_GBps": bytes_pt * N * nf / (ms * 1e-3) / 1e9}))


if __name__ == "__main__":
    main()
