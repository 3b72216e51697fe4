"""Galerkin entries of the JVIE operator N on a uniform voxel grid.

Sec. 2 defines N f = curl curl int g f with g = exp(-j k R)/(4 pi R) and the
orthonormal piecewise-constant basis p_i^alpha = alpha_hat / sqrt(V), giving
N^{ab}_{ij} = <N p_j^b, p_i^a> (Eq. op_N).  The paper takes the singular
6-D integrals from its cited work and does not print them, so this oracle uses
the following stated reading of the entries (the CUDA path uses the same
reading, written independently):

* curl curl = grad div - laplacian and (laplacian + k^2) g = -delta give
  N = I + G with  G f = (k^2 + grad div) int g f.
* Off-diagonal voxel pairs (offset d != 0, R = h |d|): one-point (midpoint)
  rule on both voxels,
      G^{ab}(d) = V (k^2 delta_ab + d_a d_b) g(R)
               = V g(R) [ (k^2 - (1 + jkR)/R^2) delta_ab
                          + (3 + 3jkR - k^2 R^2)/R^2  r_a r_b ],
  with r = d/|d| and V = h^3.
* Self term (d = 0): the field at the centre of the equal-volume sphere
  (radius a = (3V/(4 pi))^(1/3)) carrying a uniform current,
      G^{ab}(0) = delta_ab [ -1/3 + (2/3)((1 + jka) exp(-jka) - 1) ].

k is the background wavenumber k_b = k0 sqrt(eps_b): the problem is posed
relative to the cladding (Table 1 lists Si in SiO2 as 12.1/2.085).

The six unique components (Eq. sys_mat remark: N^{ab} = N^{ba}) are returned in
the order xx, xy, xz, yy, yz, zz.
"""
from __future__ import annotations

import math

import numpy as np

PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))   # xx xy xz yy yz zz
PAIR_INDEX = {(a, b): i for i, (a, b) in enumerate(PAIRS)}
PAIR_INDEX.update({(b, a): i for i, (a, b) in enumerate(PAIRS)})


def pair_index(a: int, b: int) -> int:
    return PAIR_INDEX[(a, b)]


def self_term(h: float, k: float) -> complex:
    """G^{aa}(0) for the equal-volume sphere (see module docstring)."""
    a = (3.0 * h ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0)
    ka = k * a
    return -1.0 / 3.0 + (2.0 / 3.0) * ((1.0 + 1j * ka) * np.exp(-1j * ka) - 1.0)


def entries(dx, dy, dz, h: float, k: float) -> np.ndarray:
    """G^{ab}(d) for integer voxel offsets d = (dx, dy, dz) (broadcast arrays).

    Returns complex128 of shape (6,) + broadcast shape, components in PAIRS
    order.  Zero offsets get the self term on the diagonal components.
    """
    dx, dy, dz = np.broadcast_arrays(np.asarray(dx, dtype=np.float64),
                                     np.asarray(dy, dtype=np.float64),
                                     np.asarray(dz, dtype=np.float64))
    shape = dx.shape
    out = np.zeros((6,) + shape, dtype=np.complex128)
    d2 = dx * dx + dy * dy + dz * dz
    off = d2 > 0
    dist = np.sqrt(np.where(off, d2, 1.0))
    R = h * dist
    V = h ** 3
    g = np.exp(-1j * k * R) / (4.0 * math.pi * R)
    c_delta = k * k - (1.0 + 1j * k * R) / (R * R)
    c_rr = (3.0 + 3.0j * k * R - (k * R) ** 2) / (R * R)
    rhat = (dx / dist, dy / dist, dz / dist)
    for i, (a, b) in enumerate(PAIRS):
        val = c_rr * rhat[a] * rhat[b]
        if a == b:
            val = val + c_delta
        out[i] = np.where(off, V * g * val, 0.0)
    st = self_term(h, k)
    for i, (a, b) in enumerate(PAIRS):
        if a == b:
            out[i] = np.where(off, out[i], st)
    return out


def parity(a: int, b: int, axis: int) -> int:
    """Sign of G^{ab} under reversal of the offset along ``axis``: the
    r_a r_b factor is odd in an axis iff exactly one of a, b equals it."""
    return -1 if ((a == axis) != (b == axis)) else 1
