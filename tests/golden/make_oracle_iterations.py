"""Write oracle_iterations.json: the FP64 CPU oracle's own iteration count,
energy and final residual for a full solve of each benchmarked workload
(PCG_C, Algorithm 2, to ||H phi - lambda phi||_inf < 1e-8 from the seeded
initial guess).  The benchmark's CPU legs time bounded samples of oracle
iterations and scale them by these counts, so that a reported oracle
throughput is the oracle's own full solve, not the GPU's iteration count.

Run from the repository root:  python tests/golden/make_oracle_iterations.py [workload ...]
Calls only oracle/ and the seeded input generators.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import gpe_oracle as O  # noqa: E402
from paper_1611_02045_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "oracle_iterations.json")


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    for name in names:
        w = I.workload(name)
        prob = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
        t0 = time.perf_counter()
        _, rep = O.pcg_solve(prob, w["phi0"], O.SolveOptions(tol_res_inf=1e-8, max_iter=100000))
        data[name] = {"status": rep["status"], "iters": rep["iters"], "E": rep["E"], "res_inf": rep["res_inf"],
                      "seconds_1thread": round(time.perf_counter() - t0, 1),
                      "note": "FP64 numpy oracle, tol_res_inf 1e-8, default options"}
        print(name, data[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=2)
            fh.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["fast256_2d"])
