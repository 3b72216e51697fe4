"""Chan-Olkin 2-level circulant preconditioner of one box (Sec. 4, the
paragraph after the C_B^{-1} display; used for the disk box of Sec. 5.3.1).

With the unknowns of a box ordered [alpha][z][y][x], the 1-level construction
turns the box operator into the per-frequency blocks D_f (Eq. Di).  When M~
is also y-invariant, every D_f consists of q = 3 nzb block rows and columns
(index (alpha, z)) whose p x p blocks (p = nyb, index y) are Toeplitz: the
entry between rows (a, z, y) and columns (b, z', y') depends on y - y' only.
The 2-level preconditioner C_B2 repeats the circulant step on those blocks:
each Toeplitz y-block of D_f is replaced by its Chan circulant (Eq. Chan),
and the y-DFT diagonalises the result, leaving one dense 3 nzb x 3 nzb block
per frequency pair (f, g):

  D_{f,g}[(a,z), (b,z')] = delta - M~_z (delta + lambda_{f,g}^{ab}(z - z')),

where lambda_{f,g}^{ab}(dz) is the y-DFT at g of the Chan vector of the
y-Toeplitz sequence dy -> lambda_f^{ab}(dy, dz) (lambda_f from the 1-level
step, Eq. Chan along x and the x-DFT).  The identity part of D_f sits on the
dy = 0 diagonal only and is its own Chan circulant.  The inverse is
C_B2^{-1} = F^{-1} P^T diag(D_{f,g}^{-1}) P F with F the 2-D DFT over (y, x)
of every (alpha, z) plane.  Cost O(nx ny nz^3) against O(nx (ny nz)^3).

Reading (not stated in the paper): M~ is homogenised over each z-plane of the
box (``homogenize.homogenize_plane``), so that the y-blocks are Toeplitz.
Memory reduction (Sec. 5.1.1) is a 1-level device and is not applied here.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import circulant, greens, homogenize
from .precond import chan_eigs


def chan2_eigs(nxb: int, nyb: int, nzb: int, h: float, k: float) -> np.ndarray:
    """lambda2[c, dz + nzb - 1, g, f]: the second circulant level applied to
    the 1-level eigenvalues lambda[c, dz, dy, f] along dy, then the y-DFT."""
    lam = chan_eigs(nxb, nyb, nzb, h, k)            # [c][dz][dy + nyb - 1][f]
    out = np.empty((6, 2 * nzb - 1, nyb, nxb), dtype=np.complex128)
    j = np.arange(nyb)
    for c in range(6):
        for iz in range(2 * nzb - 1):
            for f in range(nxb):
                seq = lam[c, iz, :, f]               # dy = -(nyb-1) .. nyb-1
                t_pos = seq[nyb - 1 + j]              # t_j,  j = 0..nyb-1
                t_neg = seq[nyb - 1 - j]              # t_{-j}
                cvec = circulant.chan_closed_form(t_pos, t_neg)
                out[c, iz, :, f] = circulant.eigenvalues(cvec)
    return out


def block_order(nzb: int):
    """Row index p -> (alpha, z) for the [alpha][z] ordering of D_{f,g}."""
    p = np.arange(3 * nzb)
    return np.divmod(p, nzb)


def assemble_blocks2(Mt: np.ndarray, lam2: np.ndarray, nxb: int, nyb: int, nzb: int) -> np.ndarray:
    """D_{f,g} for every (f, g) as an array (nxb, nyb, 3 nzb, 3 nzb)."""
    a, z = block_order(nzb)
    m2 = len(a)
    cidx = np.array([[greens.pair_index(a[p], a[q]) for q in range(m2)] for p in range(m2)])
    dz = z[:, None] - z[None, :] + nzb - 1
    L = lam2[cidx, dz]                              # (m2, m2, nyb, nxb)
    L = np.transpose(L, (3, 2, 0, 1))               # (nxb, nyb, m2, m2)
    Mp = Mt[z]
    D = -Mp[None, None, :, None] * L
    D[:, :, np.arange(m2), np.arange(m2)] += 1.0 - Mp[None, None, :]
    return D


class TwoLevelBoxPreconditioner:
    """C_B2^{-1} of one box (no memory reduction)."""

    levels = 2

    def __init__(self, box, M_full: np.ndarray, h: float, k: float,
                 variant: int = homogenize.REAL_MEAN):
        self.box = tuple(int(v) for v in box[:6])
        x0, y0, z0, nxb, nyb, nzb = self.box
        self.n = nxb
        self.m2 = 3 * nzb
        Mb = M_full[z0:z0 + nzb, y0:y0 + nyb, x0:x0 + nxb]
        self.Mt = homogenize.homogenize_plane(Mb, variant)
        self.lam2 = chan2_eigs(nxb, nyb, nzb, h, k)
        self.D = assemble_blocks2(self.Mt, self.lam2, nxb, nyb, nzb)
        self.lu = [[sla.lu_factor(self.D[f, g]) for g in range(nyb)] for f in range(nxb)]

    def apply_box(self, r_box: np.ndarray) -> np.ndarray:
        """C_B2^{-1} r for r_box of shape [3][nzb][nyb][nxb]."""
        x0, y0, z0, nxb, nyb, nzb = self.box
        R = np.fft.fft2(r_box.reshape(self.m2, nyb, nxb), axes=(1, 2))   # F over (y, x)
        Z = np.empty_like(R)
        for f in range(nxb):                                              # diag(D_{f,g}^{-1})
            for g in range(nyb):
                Z[:, g, f] = sla.lu_solve(self.lu[f][g], R[:, g, f])
        return np.fft.ifft2(Z, axes=(1, 2)).reshape(r_box.shape)         # F^{-1}


def homogenized_box_matrix2(box, M_full, h, k, variant) -> np.ndarray:
    """Dense A~2 = I - M~ (I + G) of one box with the plane-homogenised M~,
    [alpha][z][y][x] ordering (tiny boxes only)."""
    from .operator import dense_matrix
    x0, y0, z0, nxb, nyb, nzb = box[:6]
    Mt = homogenize.homogenize_plane(M_full[z0:z0 + nzb, y0:y0 + nyb, x0:x0 + nxb], variant)
    Mgrid = np.broadcast_to(Mt[:, None, None], (nzb, nyb, nxb))
    return dense_matrix(nxb, nyb, nzb, h, k, np.ascontiguousarray(Mgrid))


def chan2_block_dense(A_box: np.ndarray, m2: int, nyb: int, nxb: int) -> np.ndarray:
    """C_B2 from its definition: every (ny nx) x (ny nx) block of the dense
    matrix (block index (alpha, z), inner index [y][x]) replaced by its
    Frobenius-nearest 2-level circulant (``circulant.chan2_from_matrix``)."""
    s = nyb * nxb
    C = np.zeros_like(A_box)
    for p in range(m2):
        for q in range(m2):
            T = A_box[p * s:(p + 1) * s, q * s:(q + 1) * s]
            C[p * s:(p + 1) * s, q * s:(q + 1) * s] = circulant.circulant2(
                circulant.chan2_from_matrix(T, nyb, nxb))
    return C
