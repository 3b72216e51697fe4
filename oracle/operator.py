"""The discrete JVIE system (I - M N) w = M e_inc (Sec. 2, Eq. discrete_form).

Unknowns are ordered [alpha][z][y][x] (x fastest), alpha = x, y, z, matching
the block layout of Eq. sys_mat: three component blocks, each 3-level Toeplitz.
The right-hand side omits the scalar j omega eps0 (the unknown is the
normalised current w = j / (j omega eps0)).

Two matvecs:
* ``dense_matrix`` assembles A = I - diag(M)(I + G) entry by entry from the
  generator reading in ``oracle.greens`` (tiny grids only).
* ``fft_matvec`` applies the same A through the zero-padded circulant
  embedding of each 3-level Toeplitz block (the O(n log n) product the paper
  uses, Sec. 1 and Sec. 2), with numpy's FFT as the transform step.
"""
from __future__ import annotations

import math

import numpy as np

from . import greens


def material(eps: np.ndarray, eps_bg: float) -> np.ndarray:
    """M = (eps_r - 1)/eps_r with eps_r relative to the background (Sec. 2,
    after Eq. JVIE; Table 1 'Si in SiO2')."""
    er = eps / eps_bg
    return (er - 1.0) / er


def background_k(k0: float, eps_bg: float) -> float:
    return k0 * math.sqrt(eps_bg)


def rhs(eps: np.ndarray, eps_bg: float, e_inc: np.ndarray) -> np.ndarray:
    """b = M e_inc per component (Eq. discrete_form without j omega eps0)."""
    return material(eps, eps_bg)[None] * e_inc


def dense_matrix(nx: int, ny: int, nz: int, h: float, k: float, M: np.ndarray) -> np.ndarray:
    """A = I - diag(M,M,M) (I + G) as a dense (3N x 3N) complex128 matrix."""
    N = nx * ny * nz
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix = ix.ravel(); iy = iy.ravel(); iz = iz.ravel()
    dx = ix[:, None] - ix[None, :]
    dy = iy[:, None] - iy[None, :]
    dz = iz[:, None] - iz[None, :]
    G6 = greens.entries(dx, dy, dz, h, k)          # (6, N, N)
    Nmat = np.zeros((3 * N, 3 * N), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            Nmat[a * N:(a + 1) * N, b * N:(b + 1) * N] = G6[greens.pair_index(a, b)]
    Nmat += np.eye(3 * N)
    Mv = np.tile(M.ravel(), 3)
    return np.eye(3 * N) - Mv[:, None] * Nmat


def embedding_lengths(nx: int, ny: int, nz: int):
    """Circulant embedding lengths: 2n per axis (any length >= 2n-1 is exact)."""
    return 2 * nx, 2 * ny, 2 * nz


def generator_spectra(nx, ny, nz, h, k, L=None, Py=None, Pz=None) -> np.ndarray:
    """FFT of each of the 6 generators placed in a circulant of size
    (Pz, Py, L): offset d goes to index d mod P, unused indices are zero."""
    L0, Py0, Pz0 = embedding_lengths(nx, ny, nz)
    L = L0 if L is None else L
    Py = Py0 if Py is None else Py
    Pz = Pz0 if Pz is None else Pz
    assert L >= 2 * nx - 1 and Py >= 2 * ny - 1 and Pz >= 2 * nz - 1
    dxs = np.arange(-(nx - 1), nx)
    dys = np.arange(-(ny - 1), ny)
    dzs = np.arange(-(nz - 1), nz)
    DZ, DY, DX = np.meshgrid(dzs, dys, dxs, indexing="ij")
    G6 = greens.entries(DX, DY, DZ, h, k)
    spec = np.zeros((6, Pz, Py, L), dtype=np.complex128)
    iz = np.mod(DZ, Pz); iy = np.mod(DY, Py); ix = np.mod(DX, L)
    for c in range(6):
        buf = np.zeros((Pz, Py, L), dtype=np.complex128)
        buf[iz, iy, ix] = G6[c]
        spec[c] = np.fft.fftn(buf)
    return spec


def fft_matvec(x: np.ndarray, M: np.ndarray, spec: np.ndarray) -> np.ndarray:
    """y = x - M (x + G x) with G x from the circulant embedding.

    x: complex128 [3][nz][ny][nx]; spec: generator_spectra(...).
    """
    _, nz, ny, nx = x.shape
    _, Pz, Py, L = spec.shape
    X = np.empty((3, Pz, Py, L), dtype=np.complex128)
    for b in range(3):
        pad = np.zeros((Pz, Py, L), dtype=np.complex128)
        pad[:nz, :ny, :nx] = x[b]
        X[b] = np.fft.fftn(pad)
    y = np.empty_like(x)
    for a in range(3):
        acc = np.zeros((Pz, Py, L), dtype=np.complex128)
        for b in range(3):
            acc += spec[greens.pair_index(a, b)] * X[b]
        Gx = np.fft.ifftn(acc)[:nz, :ny, :nx]
        y[a] = x[a] - M * (x[a] + Gx)
    return y


def dense_matvec(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    return (A @ x.ravel()).reshape(x.shape)


def matrix_row(row: int, nx, ny, nz, h, k, M: np.ndarray) -> np.ndarray:
    """One row of A (length 3N), evaluated directly from the generator
    reading; used to check large-grid matvecs at sampled outputs."""
    N = nx * ny * nz
    a, v = divmod(row, N)
    iz0, rem = divmod(v, nx * ny)
    iy0, ix0 = divmod(rem, nx)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    G6 = greens.entries(ix0 - ix, iy0 - iy, iz0 - iz, h, k)
    out = np.zeros(3 * N, dtype=np.complex128)
    Mi = M.ravel()[v]
    for b in range(3):
        blk = G6[greens.pair_index(a, b)].ravel()
        out[b * N:(b + 1) * N] = -Mi * blk
    out[a * N + v] += 1.0 - Mi
    return out
