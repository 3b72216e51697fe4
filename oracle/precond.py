"""Chan-Olkin 1-level circulant preconditioner, its block-diagonal
(partitioned) form and its memory reduction (Sec. 4, Sec. 5.1.1, Sec. 5.3).

For one box of nxb x nyb x nzb voxels, order the box unknowns
[alpha][z][y][x].  The box operator A~ = I - M~ (I + G) with an x-invariant M~
(Sec. 5.2) is Toeplitz-block: m = 3 nyb nzb blocks per side, each an
nxb x nxb Toeplitz matrix along x.  Its circulant-block approximation C_B
replaces every block by its Chan circulant (Eq. Chan), and
C_B^{-1} = F^{-1} P^T diag(D_1^{-1} .. D_n^{-1}) P F (Eq. Di and the
following display): an x-DFT of every line, one dense m x m solve per
frequency, and an inverse x-DFT.

Because C(.) is linear, C(I) = I and M~ is diagonal and x-invariant,
  D_f[p, q] = delta_pq - M~_p (delta_pq + lambda_f^{pq}),
where lambda^{pq} = F c^{pq} and c^{pq} is the Chan vector of the Toeplitz
block of G between rows p = (a, z, y) and columns q = (b, z', y').

Memory reduction (Sec. 5.1.1, Eqs. proxy1 and proxy2): v_f is the (1, c*)
entry of D_f with c* = ceil(nyb/2) ceil(nzb/2) (1-based, taken literally as a
column index), v^ = |v| / ||v||_inf; D_f is kept where v^_f > tau and every
other frequency uses the central block D_{ceil(nxb/2)} (1-based).  Reading:
v^ is invariant to the constant factor -M~_0 that multiplies the G-part of
that off-diagonal entry, so v_f is taken as lambda_f^{(0, c*)}, which gives the
paper's v^ whenever M~_0 != 0 and stays defined when the first voxel of the
box is cladding (M~_0 = 0).  If c* = 0 (a 1-2 voxel cross-section) the entry is
diagonal and D_f[0, 0] itself is used.

Partitioning (Sec. 5.3): the preconditioner is block-diagonal over the boxes,
each block the 1-level (or, for a box given as (x0, y0, z0, nx, ny, nz, 2),
the 2-level, ``oracle.precond2``) preconditioner of its box; unknowns outside
every box get the identity.  Boxes must not overlap.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg as sla

from . import circulant, greens, homogenize
from .operator import material


def box_order(nyb: int, nzb: int):
    """Row index p -> (alpha, z, y) for the [alpha][z][y] ordering."""
    m = 3 * nyb * nzb
    p = np.arange(m)
    a, rem = np.divmod(p, nyb * nzb)
    z, y = np.divmod(rem, nyb)
    return a, z, y


def chan_eigs(nxb: int, nyb: int, nzb: int, h: float, k: float) -> np.ndarray:
    """lambda[c, dz + nzb - 1, dy + nyb - 1, f] for the 6 generator pairs and
    every transverse offset: the DFT of the Chan vector (Eq. Chan) of the
    x-Toeplitz line t_i = G^c(i, dy, dz), i in (-nxb, nxb)."""
    n = nxb
    dys = np.arange(-(nyb - 1), nyb)
    dzs = np.arange(-(nzb - 1), nzb)
    i = np.arange(n)
    out = np.zeros((6, len(dzs), len(dys), n), dtype=np.complex128)
    for iz, dz in enumerate(dzs):
        for iy, dy in enumerate(dys):
            t_pos = greens.entries(i, dy, dz, h, k)      # t_i,  i = 0..n-1
            t_neg = greens.entries(-i, dy, dz, h, k)     # t_{-i}
            for c in range(6):
                cvec = circulant.chan_closed_form(t_pos[c], t_neg[c])
                out[c, iz, iy] = circulant.eigenvalues(cvec)
    return out


def assemble_blocks(Mt: np.ndarray, lam: np.ndarray, nxb: int, nyb: int, nzb: int) -> np.ndarray:
    """D_f for f = 0..nxb-1 as an array (nxb, m, m)."""
    a, z, y = box_order(nyb, nzb)
    m = len(a)
    cidx = np.array([[greens.pair_index(a[p], a[q]) for q in range(m)] for p in range(m)])
    dz = z[:, None] - z[None, :] + nzb - 1
    dy = y[:, None] - y[None, :] + nyb - 1
    L = lam[cidx, dz, dy, :]                       # (m, m, nxb)
    L = np.moveaxis(L, 2, 0)                        # (nxb, m, m)
    Mp = Mt[z, y]                                   # M~ per row p
    D = -Mp[None, :, None] * L
    D[:, np.arange(m), np.arange(m)] += 1.0 - Mp[None, :]
    return D


def proxy(lam: np.ndarray, Mt: np.ndarray, nxb: int, nyb: int, nzb: int) -> np.ndarray:
    """v^ of Eqs. proxy1-proxy2 under the reading in the module docstring."""
    cstar = int(math.ceil(nyb / 2) * math.ceil(nzb / 2)) - 1   # 0-based column
    a, z, y = box_order(nyb, nzb)
    if cstar == 0:
        v = 1.0 - Mt[0, 0] * (1.0 + lam[greens.pair_index(0, 0), nzb - 1, nyb - 1, :])
    else:
        c = greens.pair_index(a[0], a[cstar])
        v = lam[c, z[0] - z[cstar] + nzb - 1, y[0] - y[cstar] + nyb - 1, :]
    av = np.abs(v)
    mx = av.max()
    return av / mx if mx > 0 else np.ones_like(av)


class BoxPreconditioner:
    """1-level (optionally reduced) circulant preconditioner of one box."""

    def __init__(self, box, M_full: np.ndarray, h: float, k: float,
                 variant: int = homogenize.REAL_MEAN, tau: float = 0.0):
        self.box = tuple(int(v) for v in box[:6])
        x0, y0, z0, nxb, nyb, nzb = self.box
        self.n = nxb
        self.m = 3 * nyb * nzb
        Mb = M_full[z0:z0 + nzb, y0:y0 + nyb, x0:x0 + nxb]
        self.Mt = homogenize.homogenize(Mb, variant)
        self.lam = chan_eigs(nxb, nyb, nzb, h, k)
        self.D = assemble_blocks(self.Mt, self.lam, nxb, nyb, nzb)
        self.tau = tau
        self.vhat = proxy(self.lam, self.Mt, nxb, nyb, nzb)
        self.rep = int(math.ceil(nxb / 2)) - 1
        if tau > 0:
            self.kept = np.nonzero(self.vhat > tau)[0]
        else:
            self.kept = np.arange(nxb)
        keep = np.zeros(nxb, dtype=bool)
        keep[self.kept] = True
        self.keep_mask = keep
        self.lu = {}
        for f in list(self.kept) + [self.rep]:
            if f not in self.lu:
                self.lu[int(f)] = sla.lu_factor(self.D[f])

    def block_for(self, f: int) -> int:
        return int(f) if self.keep_mask[f] else self.rep

    def apply_box(self, r_box: np.ndarray) -> np.ndarray:
        """C_B^{-1} r for r_box of shape [3][nzb][nyb][nxb]."""
        x0, y0, z0, nxb, nyb, nzb = self.box
        lines = r_box.reshape(self.m, nxb)
        R = np.fft.fft(lines, axis=1)               # F (x-DFT of every line)
        Z = np.empty_like(R)
        for f in range(nxb):                        # P, diag(D_f^{-1}), P^T
            Z[:, f] = sla.lu_solve(self.lu[self.block_for(f)], R[:, f])
        z = np.fft.ifft(Z, axis=1)                   # F^{-1}
        return z.reshape(r_box.shape)

    def dense_inverse_apply(self, r_box: np.ndarray) -> np.ndarray:
        """Same operator through the dense per-frequency matrix D_f^{-1} (no
        LU reuse); used by tests only."""
        x0, y0, z0, nxb, nyb, nzb = self.box
        R = np.fft.fft(r_box.reshape(self.m, nxb), axis=1)
        Z = np.empty_like(R)
        for f in range(nxb):
            Z[:, f] = np.linalg.solve(self.D[self.block_for(f)], R[:, f])
        return np.fft.ifft(Z, axis=1).reshape(r_box.shape)


class Preconditioner:
    """Block-diagonal (partitioned) circulant preconditioner (Sec. 5.3)."""

    def __init__(self, nx, ny, nz, h, k, M: np.ndarray, boxes: Optional[Sequence] = None,
                 variant: int = homogenize.REAL_MEAN, tau: float = 0.0):
        boxes = list(boxes) if boxes else [(0, 0, 0, nx, ny, nz)]
        self.shape = (3, nz, ny, nx)
        self.boxes = []
        for b in boxes:
            if len(b) > 6 and int(b[6]) == 2:
                from .precond2 import TwoLevelBoxPreconditioner
                self.boxes.append(TwoLevelBoxPreconditioner(b, M, h, k, variant))
            else:
                self.boxes.append(BoxPreconditioner(b, M, h, k, variant, tau))

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = r.copy()                                   # identity outside the boxes
        for bp in self.boxes:
            x0, y0, z0, nxb, nyb, nzb = bp.box
            sl = (slice(None), slice(z0, z0 + nzb), slice(y0, y0 + nyb), slice(x0, x0 + nxb))
            z[sl] = bp.apply_box(r[sl])
        return z


def chan_block_dense(A_box: np.ndarray, m: int, n: int) -> np.ndarray:
    """C_B from its definition: the Chan circulant (Frobenius-nearest,
    wrapped-diagonal mean) of every n x n block of the dense m n x m n matrix
    A_box in [block][x] ordering (Sec. 4, circulant-block approximation)."""
    C = np.zeros_like(A_box)
    for p in range(m):
        for q in range(m):
            T = A_box[p * n:(p + 1) * n, q * n:(q + 1) * n]
            C[p * n:(p + 1) * n, q * n:(q + 1) * n] = circulant.circulant(
                circulant.chan_from_matrix(T))
    return C


def homogenized_box_matrix(box, M_full, h, k, variant) -> np.ndarray:
    """Dense A~ = I - M~ (I + G) of one box, [alpha][z][y][x] ordering (tiny
    boxes only)."""
    from .operator import dense_matrix
    x0, y0, z0, nxb, nyb, nzb = box
    Mt = homogenize.homogenize(M_full[z0:z0 + nzb, y0:y0 + nyb, x0:x0 + nxb], variant)
    Mgrid = np.broadcast_to(Mt[:, :, None], (nzb, nyb, nxb))
    return dense_matrix(nxb, nyb, nzb, h, k, np.ascontiguousarray(Mgrid))
