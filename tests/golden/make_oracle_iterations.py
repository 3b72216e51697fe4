"""Write tests/golden/oracle_iterations.json: iteration counts and timings of
the CPU oracle's preconditioned GMRES(50) (right preconditioning, real-mean
homogenisation, reduction tau = 1e-3) on the benchmark workloads.  Calls only
oracle/ and the shared input generators.  bench.py uses the counts to scale
its bounded oracle sample to a full solve.

Usage: python tests/golden/make_oracle_iterations.py [workload ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solve as osolve                  # noqa: E402
from paper_1903_07884_gb300 import inputs          # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")
WORKLOADS = {
    "small_straight_64x8x4": inputs.workload_small_straight,
    "long_straight_1024x16x8": inputs.workload_long_straight,
}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p = WORKLOADS[name]()
        for tol in (1e-9,):
            t0 = time.perf_counter()
            s = osolve.iterative_solve(p, tol=tol, tau=1e-3)
            data.setdefault(name, {})[f"{tol:g}"] = {
                "iters": s.iters, "relres": s.relres, "t_setup_s": s.t_setup, "t_solve_s": s.t_solve,
                "cores": len(os.sched_getaffinity(0)), "wall_s": time.perf_counter() - t0}
            print(name, tol, data[name][f"{tol:g}"], flush=True)
            json.dump(data, open(OUT, "w"), indent=2)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
