"""Batched parameter sweep benchmark: many independent 2D ground states in one
graph launch (gpe_batch_solve) against the same instances solved one at a
time (gpe_pcg_solve, FP64 or mixed).

    python sweepbench.py --count 96 --steps 2
    python sweepbench.py --count 96 --single fp64

Instances: inputs.sweep_instances (grids 128^2 / 256^2 / 512^2 on [-16,16]^2,
omega ~ U[0, 0.95], eta in {100, 250, 500, 1000}, kappa in {0, 0.05}).
Prints one JSON line.  Times are CUDA events on the stream the work runs on,
with the initial guesses already on the device.
"""
from __future__ import annotations

import argparse
import json
import statistics


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=96)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--single", choices=["none", "fp64", "mixed"], default="none",
                    help="also time every instance solved alone, in this precision")
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default pass-kernel plans")
    a = ap.parse_args()

    import torch

    from paper_1611_02045_gb300 import build, gpe, inputs as I
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    insts = I.sweep_instances(a.count)
    arrays = [I.sweep_arrays(w) for w in insts]
    specs = [dict(n=w["n"], L=w["L"], eta=w["eta"], omega=w["omega"], V=V, prec=gpe.GPE_MIXED)
             for w, (V, _) in zip(insts, arrays)]
    phi0 = [torch.from_numpy(p.copy()).to(dev) for _, p in arrays]
    opts = gpe.solve_opts_default()
    opts.max_iter = a.max_iter

    out = dict(bench="sweep", count=a.count, grids=sorted({w["n"][0] for w in insts}), autotune=not a.no_autotune)
    with gpe.Batch(specs) as B:
        if not a.no_autotune:
            B.autotune(iters=10)  # one tuning per distinct grid (process cache)
        phis = [torch.empty_like(p) for p in phi0]
        times, reps = [], None
        for k in range(a.warmup + a.steps):
            for p, q in zip(phis, phi0):
                p.copy_(q)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s, reps = B.solve(phis, opts)
            e1.record(stream)
            e1.synchronize()
            if k >= a.warmup:
                times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    ok = sum(r["status"] == gpe.GPE_OK for r in reps)
    out.update(batch_ms=ms, batch_ground_states_per_s=a.count / (ms * 1e-3), converged=ok,
               iters_total=int(sum(r["iters"] for r in reps)),
               iters_by_grid={str(g): int(sum(r["iters"] for r, w in zip(reps, insts) if w["n"][0] == g))
                              for g in out["grids"]},
               max_res_inf=float(max(r["res_inf"] for r in reps)),
               fp64_completions=int(sum(r["iters_fp64"] > 0 for r in reps)),
               iters_fp64_total=int(sum(r["iters_fp64"] for r in reps)))
    if a.single != "none":
        prec = gpe.GPE_FP64 if a.single == "fp64" else gpe.GPE_MIXED
        tot, ok1, its = 0.0, 0, 0
        for w, (V, _), p0 in zip(insts, arrays, phi0):
            with gpe.Context(w["n"], w["L"], w["eta"], w["omega"], V, prec=prec) as ctx:
                if not a.no_autotune:
                    ctx.autotune(iters=10)
                phi = p0.clone()
                ctx.pcg_solve(phi.clone(), opts)  # builds the graphs
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep = ctx.pcg_solve(phi, opts)
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
                ok1 += rep["status"] == gpe.GPE_OK
                its += rep["iters"]
        out.update({f"single_{a.single}_ms": tot, f"single_{a.single}_ground_states_per_s": a.count / (tot * 1e-3),
                    f"single_{a.single}_converged": ok1, f"single_{a.single}_iters_total": its})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
