"""T. Chan's optimal circulant and its diagonalisation (Sec. 4).

* ``chan_from_matrix``: the Frobenius-nearest circulant of an n x n matrix T,
  written from its definition (minimise ||C - T||_F over circulants): c_k is
  the mean of T over the wrapped diagonal {(i, j) : (i - j) mod n = k}.
* ``chan_closed_form``: Eq. Chan for a Toeplitz T with t_{i-j} = T_ij,
  c_i = ((n - i) t_i + i t_{-(n-i)}) / n, 0 <= i <= n-1.
* ``circulant``: the matrix with c_ij = c_{(i-j) mod n} (Sec. 4).
* ``eigenvalues``: Lambda = diag(F c), C = F^{-1} Lambda F, F the DFT matrix
  F_{fk} = exp(-2 pi i f k / n) (Sec. 4, diagonalisation remark).
"""
from __future__ import annotations

import numpy as np


def chan_from_matrix(T: np.ndarray) -> np.ndarray:
    n = T.shape[0]
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = np.mod(i - j, n)
    c = np.zeros(n, dtype=np.result_type(T, np.complex128))
    for kk in range(n):
        c[kk] = T[k == kk].mean()
    return c


def chan_closed_form(t_pos: np.ndarray, t_neg: np.ndarray) -> np.ndarray:
    """t_pos[i] = t_i (i = 0..n-1), t_neg[i] = t_{-i} (i = 0..n-1, t_neg[0]
    unused).  Returns c_0..c_{n-1} by Eq. Chan."""
    n = len(t_pos)
    c = np.empty(n, dtype=np.result_type(t_pos, t_neg, np.complex128))
    c[0] = t_pos[0]
    for i in range(1, n):
        c[i] = ((n - i) * t_pos[i] + i * t_neg[n - i]) / n
    return c


def toeplitz(t_pos: np.ndarray, t_neg: np.ndarray) -> np.ndarray:
    n = len(t_pos)
    T = np.empty((n, n), dtype=np.result_type(t_pos, t_neg, np.complex128))
    for i in range(n):
        for j in range(n):
            T[i, j] = t_pos[i - j] if i >= j else t_neg[j - i]
    return T


def circulant(c: np.ndarray) -> np.ndarray:
    n = len(c)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return c[np.mod(i - j, n)]


def dft_matrix(n: int) -> np.ndarray:
    f, k = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.exp(-2j * np.pi * f * k / n)


def eigenvalues(c: np.ndarray) -> np.ndarray:
    """lambda_f = sum_k c_k exp(-2 pi i f k / n), i.e. F c."""
    return np.fft.fft(c)


def chan2_from_matrix(T: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Frobenius-nearest 2-level circulant (circulant blocks in a circulant
    block pattern) of an (n1 n2) x (n1 n2) matrix in [i1][i2] ordering, from
    its definition: c[k1, k2] is the mean of T over every entry whose index
    difference is (k1, k2) modulo (n1, n2)."""
    i1, i2 = np.divmod(np.arange(n1 * n2), n2)
    k1 = np.mod(i1[:, None] - i1[None, :], n1)
    k2 = np.mod(i2[:, None] - i2[None, :], n2)
    c = np.zeros((n1, n2), dtype=np.result_type(T, np.complex128))
    for a in range(n1):
        for b in range(n2):
            c[a, b] = T[(k1 == a) & (k2 == b)].mean()
    return c


def circulant2(c: np.ndarray) -> np.ndarray:
    """The 2-level circulant with entries c[(i1 - j1) mod n1, (i2 - j2) mod n2]."""
    n1, n2 = c.shape
    i1, i2 = np.divmod(np.arange(n1 * n2), n2)
    return c[np.mod(i1[:, None] - i1[None, :], n1), np.mod(i2[:, None] - i2[None, :], n2)]
