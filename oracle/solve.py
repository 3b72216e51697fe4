"""Reference solutions of the JVIE system (Sec. 2, Eq. discrete_form).

``dense_solve`` uses a direct LU of the dense matrix (tiny grids);
``iterative_solve`` runs the oracle GMRES on the FFT matvec, preconditioned by
the oracle's circulant preconditioner.  The solution of the linear system does
not depend on the preconditioner; it only changes the iteration count.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Optional

import numpy as np

from . import gmres as _gmres
from . import operator as op
from . import precond as pc


@dataclasses.dataclass
class OracleSolution:
    w: np.ndarray
    iters: int
    relres: float
    t_setup: float
    t_solve: float


def system(problem):
    k = op.background_k(problem.k0, problem.eps_bg)
    M = op.material(problem.eps, problem.eps_bg)
    b = op.rhs(problem.eps, problem.eps_bg, problem.e_inc)
    return k, M, b


def dense_solve(problem) -> np.ndarray:
    k, M, b = system(problem)
    A = op.dense_matrix(problem.nx, problem.ny, problem.nz, problem.h, k, M)
    return np.linalg.solve(A, b.ravel()).reshape(b.shape)


def iterative_solve(problem, tol: float = 1e-12, tau: float = 1e-3,
                    restart: int = 50, max_iter: int = 5000,
                    use_precond: bool = True) -> OracleSolution:
    t0 = time.perf_counter()
    k, M, b = system(problem)
    spec = op.generator_spectra(problem.nx, problem.ny, problem.nz, problem.h, k)
    P = None
    if use_precond:
        P = pc.Preconditioner(problem.nx, problem.ny, problem.nz, problem.h, k, M,
                              problem.boxes, problem.homog, tau)
    t1 = time.perf_counter()
    res = _gmres.gmres(lambda v: op.fft_matvec(v, M, spec), b,
                       None if P is None else P.apply, tol=tol, restart=restart,
                       max_iter=max_iter)
    t2 = time.perf_counter()
    return OracleSolution(res.x, res.iters, res.relres, t1 - t0, t2 - t1)
