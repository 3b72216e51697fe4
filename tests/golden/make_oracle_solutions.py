"""Write the CPU oracle's reference solutions of the benchmark workloads to
tests/golden/: the solution w of (I - M N) w = M e_inc (Sec. 2, Eq.
discrete_form) that the GPU solves are compared with.

* small_straight_64x8x4: direct LU of the dense matrix (oracle.solve.dense_solve).
* long_straight_1024x16x8: the oracle's right-preconditioned GMRES(50) on its
  FFT matvec to the relative residual 1e-12 (oracle.solve.iterative_solve);
  the solution does not depend on the preconditioner.  Stored whole.
* larger workloads (4096x24x8 Bragg grating, 2048x48x8 coupler at the first
  wavelength of its batch, 1.50 um): the same
  iterative solve; stored as a seeded sample of 4096 entries plus the
  solution's 2-norm and max-abs, since the whole vector (38 MB) is too large
  to keep in the repository.

Calls only oracle/ and the shared input generators (no arithmetic of the GPU
path).  The relative residual reached and the wall time go to
oracle_solutions.json.

Usage: python tests/golden/make_oracle_solutions.py [workload ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import operator as op                   # noqa: E402
from oracle import solve as osolve                  # noqa: E402
from paper_1903_07884_gb300 import inputs          # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
META = os.path.join(HERE, "oracle_solutions.json")
SAMPLE = 4096
WORKLOADS = {
    "small_straight_64x8x4": inputs.workload_small_straight,
    "long_straight_1024x16x8": inputs.workload_long_straight,
    "bragg_4096x24x8_2boxes": inputs.workload_bragg,
    "coupler_2048x48x8_2boxes_lambda1.50": lambda: inputs.workload_coupler(wavelength=1.50),
}
FULL = {"small_straight_64x8x4", "long_straight_1024x16x8"}


def sample_indices(n3: int) -> np.ndarray:
    """Seeded sorted sample of solution indices (shared by the script and the
    tests that read the sample)."""
    rng = np.random.Generator(np.random.PCG64(1234))
    return np.unique(rng.integers(0, n3, size=SAMPLE))


def main(names):
    meta = json.load(open(META)) if os.path.exists(META) else {}
    for name in names:
        p = WORKLOADS[name]()
        t0 = time.perf_counter()
        if name == "small_straight_64x8x4":
            w = osolve.dense_solve(p)
            k, M, b = osolve.system(p)
            spec = op.generator_spectra(p.nx, p.ny, p.nz, p.h, k)
            rr = float(np.linalg.norm(b - op.fft_matvec(w, M, spec)) / np.linalg.norm(b))
            iters = 0
            how = "dense LU"
        else:
            s = osolve.iterative_solve(p, tol=1e-12, tau=1e-3, max_iter=20000)
            w, rr, iters = s.w, s.relres, s.iters
            how = "oracle GMRES(50), 1-level circulant preconditioner, tol 1e-12"
        wall = time.perf_counter() - t0
        entry = {"method": how, "relres": rr, "iters": iters, "wall_s": wall,
                 "cores": len(os.sched_getaffinity(0)), "shape": list(w.shape),
                 "norm2": float(np.linalg.norm(w)), "maxabs": float(np.abs(w).max())}
        if name in FULL:
            fn = f"oracle_solution_{name}.npy"
            np.save(os.path.join(HERE, fn), w.astype(np.complex128))
            entry["file"] = fn
        else:
            idx = sample_indices(w.size)
            fn = f"oracle_solution_{name}_sample.npz"
            np.savez(os.path.join(HERE, fn), idx=idx, w=w.ravel()[idx].astype(np.complex128))
            entry["file"] = fn
            entry["sample"] = int(idx.size)
        meta[name] = entry
        print(name, entry, flush=True)
        json.dump(meta, open(META, "w"), indent=2)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
