"""Restarted GMRES with right preconditioning (the Krylov solver of Sec. 1 and
Sec. 3; the paper does not print its variant).

Textbook algorithm (Saad and Schultz): Arnoldi with modified Gram-Schmidt on
the operator A P^{-1}, complex Givens rotations to keep the Hessenberg matrix
triangular, the residual estimate |g_{j+1}|, and at each restart
x <- x + P^{-1} V_k y_k.  Stop when the true relative residual
||b - A x|| / ||b|| is at most ``tol``; the estimate only ends a cycle early.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np
import scipy.linalg as sla


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    relres: float
    converged: bool
    history: list


def givens(a: complex, b: complex):
    """Rotation [[c, s], [-conj(s), c]] (c real) mapping (a, b) to (rho, 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    r = np.hypot(abs(a), abs(b))
    c = abs(a) / r
    s = a * np.conj(b) / (abs(a) * r)
    return c, s


def gmres(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
          apply_Pinv: Optional[Callable[[np.ndarray], np.ndarray]] = None,
          tol: float = 1e-8, restart: int = 50, max_iter: int = 2000,
          x0: Optional[np.ndarray] = None) -> GmresResult:
    shape = b.shape
    bv = b.ravel()
    P = (lambda v: v) if apply_Pinv is None else (lambda v: apply_Pinv(v.reshape(shape)).ravel())
    Aop = lambda v: apply_A(v.reshape(shape)).ravel()
    x = np.zeros_like(bv) if x0 is None else x0.ravel().copy()
    bnorm = np.linalg.norm(bv)
    history = []
    if bnorm == 0:
        return GmresResult(x.reshape(shape), 0, 0.0, True, history)
    r = bv - Aop(x)
    relres = np.linalg.norm(r) / bnorm
    iters = 0
    while relres > tol and iters < max_iter:
        beta = np.linalg.norm(r)
        n = len(bv)
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            w = Aop(P(V[j]))
            for i in range(j + 1):                    # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                        # previous rotations
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or iters >= max_iter:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + P(V[:k].T @ y)
        r = bv - Aop(x)
        relres = np.linalg.norm(r) / bnorm
    return GmresResult(x.reshape(shape), iters, float(relres), bool(relres <= tol), history)
