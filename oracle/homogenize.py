"""Homogenised material operator for the preconditioner (Sec. 5.2).

The three variants of the x-invariant M~ over a box (array indices as in the
paper's M(k, l, m) with k along x):
  1. the mode of all entries of M in the box (constant M~);
  2. the arithmetic mean along x, M~(l, m) = (1/n) sum_j M(j, l, m);
  3. the real part of that mean.
Readings: n is the box's x-length (absorber slabs included); the mode is over
exact complex values, ties broken by the smallest |value| and then by the
smallest (real, imag) pair.
"""
from __future__ import annotations

import numpy as np

MODE, MEAN, REAL_MEAN = 1, 2, 3


def mode_value(values: np.ndarray) -> complex:
    vals = values.ravel()
    uniq, counts = np.unique(vals, return_counts=True)
    best = counts.max()
    cands = uniq[counts == best]
    order = sorted(cands, key=lambda v: (abs(v), v.real, v.imag))
    return complex(order[0])


def homogenize(M_box: np.ndarray, variant: int) -> np.ndarray:
    """M_box: complex [nz][ny][nx] over the box.  Returns M~ as [nz][ny]."""
    nz, ny, nx = M_box.shape
    if variant == MODE:
        return np.full((nz, ny), mode_value(M_box), dtype=np.complex128)
    mean = M_box.sum(axis=2) / nx
    if variant == MEAN:
        return mean.astype(np.complex128)
    if variant == REAL_MEAN:
        return mean.real.astype(np.complex128)
    raise ValueError(f"unknown homogenisation variant {variant}")


def homogenize_plane(M_box: np.ndarray, variant: int) -> np.ndarray:
    """M~ for the 2-level preconditioner (Sec. 4, the 2-level paragraph, and
    Sec. 5.3.1): the second circulant level needs an operator that is
    Toeplitz along y as well, so M~ is made invariant in x and y.  Reading:
    the same three variants, taken over each z-plane of the box (mode over the
    whole box; mean over the nx ny entries of a plane; real part of that
    mean).  Returns M~ as [nz]."""
    nz, ny, nx = M_box.shape
    if variant == MODE:
        return np.full(nz, mode_value(M_box), dtype=np.complex128)
    mean = M_box.reshape(nz, ny * nx).sum(axis=1) / (nx * ny)
    if variant == MEAN:
        return mean.astype(np.complex128)
    if variant == REAL_MEAN:
        return mean.real.astype(np.complex128)
    raise ValueError(f"unknown homogenisation variant {variant}")
