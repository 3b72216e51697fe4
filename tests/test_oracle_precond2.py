"""Pins for the oracle's 2-level circulant preconditioner (Sec. 4, the
2-level paragraph; Sec. 5.3.1, blocked-circulant with a 2-level box)."""
import math

import numpy as np
import pytest

from oracle import circulant, gmres, homogenize
from oracle import operator as op
from oracle import precond as pc
from oracle import precond2 as pc2
from paper_1903_07884_gb300 import inputs

H = 0.05
K0 = 2 * math.pi / 1.55


def _M(nx, ny, nz, seed):
    return op.material(inputs.random_permittivity(nz, ny, nx, seed=seed), 1.0)


def _rng_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n1,n2", [(1, 1), (1, 4), (3, 1), (3, 4), (4, 5)])
def test_chan2_is_frobenius_nearest_2level_circulant(n1, n2):
    """chan2_from_matrix gives a 2-level circulant; it reproduces a 2-level
    circulant exactly; no 2-level circulant perturbation gets closer to T."""
    rng = np.random.default_rng(n1 * 10 + n2)
    T = _rng_c(rng, n1 * n2, n1 * n2)
    C = circulant.circulant2(circulant.chan2_from_matrix(T, n1, n2))
    # shift invariance: C[i + s, j + s] = C[i, j] for cyclic 2-level shifts
    i1, i2 = np.divmod(np.arange(n1 * n2), n2)
    for s1 in range(n1):
        for s2 in range(n2):
            perm = ((i1 + s1) % n1) * n2 + (i2 + s2) % n2
            np.testing.assert_allclose(C[np.ix_(perm, perm)], C, atol=1e-14)
    c0 = _rng_c(rng, n1, n2)
    E = circulant.circulant2(c0)
    np.testing.assert_allclose(circulant.circulant2(circulant.chan2_from_matrix(E, n1, n2)), E, atol=1e-14)
    base = np.linalg.norm(T - C)
    for _ in range(5):
        P = circulant.circulant2(1e-3 * _rng_c(rng, n1, n2))
        assert np.linalg.norm(T - (C + P)) > base


def test_chan2_equals_level_by_level_chan():
    """Chan and Olkin: the 2-level optimal circulant of a matrix is the
    1-level optimal circulant taken first inside every block (level 2) and
    then over the block pattern (level 1)."""
    n1, n2 = 3, 4
    rng = np.random.default_rng(5)
    T = _rng_c(rng, n1 * n2, n1 * n2)
    inner = np.zeros_like(T)
    for a in range(n1):
        for b in range(n1):
            blk = T[a * n2:(a + 1) * n2, b * n2:(b + 1) * n2]
            inner[a * n2:(a + 1) * n2, b * n2:(b + 1) * n2] = circulant.circulant(circulant.chan_from_matrix(blk))
    # level 1: entry (i2, j2) of block (a, b) replaced by the wrapped-diagonal mean over blocks
    outer = np.zeros_like(T)
    for i2 in range(n2):
        for j2 in range(n2):
            S = inner[i2::n2, j2::n2]                       # n1 x n1 matrix of that entry
            outer[i2::n2, j2::n2] = circulant.circulant(circulant.chan_from_matrix(S))
    C = circulant.circulant2(circulant.chan2_from_matrix(T, n1, n2))
    np.testing.assert_allclose(outer, C, atol=1e-14)


SHAPES = [(3, 2, 1), (4, 3, 2), (5, 4, 1), (2, 5, 2), (1, 3, 2), (4, 1, 2), (3, 3, 3)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_blocks2_match_dense_definition(shape, variant):
    """D_{f,g} from the level-by-level closed form (Eq. Chan twice, 2-D DFT)
    equal the 2-D DFT of the Frobenius-nearest 2-level circulants of the dense
    plane-homogenised box matrix."""
    nx, ny, nz = shape
    M = _M(nx, ny, nz, seed=3 * nx + 5 * ny + 7 * nz)
    box = (0, 0, 0, nx, ny, nz, 2)
    bp = pc2.TwoLevelBoxPreconditioner(box, M, H, K0, variant)
    A = pc2.homogenized_box_matrix2(box, M, H, K0, variant)
    m2, s = 3 * nz, ny * nx
    D_def = np.zeros((nx, ny, m2, m2), dtype=complex)
    for p in range(m2):
        for q in range(m2):
            c = circulant.chan2_from_matrix(A[p * s:(p + 1) * s, q * s:(q + 1) * s], ny, nx)
            D_def[:, :, p, q] = np.fft.fft2(c).T                 # [g][f] -> [f][g]
    np.testing.assert_allclose(bp.D, D_def, atol=1e-13)


@pytest.mark.parametrize("shape", [(4, 3, 2), (5, 4, 1), (3, 3, 3), (6, 4, 1)])
def test_apply2_equals_dense_solve(shape):
    nx, ny, nz = shape
    M = _M(nx, ny, nz, seed=11 + nx)
    box = (0, 0, 0, nx, ny, nz, 2)
    bp = pc2.TwoLevelBoxPreconditioner(box, M, H, K0, 3)
    C = pc2.chan2_block_dense(pc2.homogenized_box_matrix2(box, M, H, K0, 3), 3 * nz, ny, nx)
    r = _rng_c(np.random.default_rng(1), 3, nz, ny, nx)
    np.testing.assert_allclose(bp.apply_box(r).ravel(), np.linalg.solve(C, r.ravel()), rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(6, 4, 2), (5, 5, 1), (4, 7, 2)])
def test_symmetry_S2(shape):
    """Generator parity in x and y: D_{n-f,g} = Sx D_{f,g} Sx and
    D_{f,ny-g} = Sy D_{f,g} Sy (S = -1 on the x- resp. y-component rows)."""
    nx, ny, nz = shape
    bp = pc2.TwoLevelBoxPreconditioner((0, 0, 0, nx, ny, nz, 2), _M(nx, ny, nz, 2), H, K0, 2)
    a, _ = pc2.block_order(nz)
    Sx = np.where(a == 0, -1.0, 1.0)
    Sy = np.where(a == 1, -1.0, 1.0)
    for f in range(nx):
        for g in range(ny):
            np.testing.assert_allclose(bp.D[(nx - f) % nx, g], Sx[:, None] * bp.D[f, g] * Sx[None, :], atol=1e-13)
            np.testing.assert_allclose(bp.D[f, (ny - g) % ny], Sy[:, None] * bp.D[f, g] * Sy[None, :], atol=1e-13)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_two_level_with_one_y_voxel_is_one_level(variant):
    """With ny = 1 the second level is trivial and the plane homogenisation is
    the x homogenisation, so C_B2 = C_B."""
    nx, ny, nz = 6, 1, 3
    M = _M(nx, ny, nz, 9)
    r = _rng_c(np.random.default_rng(2), 3, nz, ny, nx)
    one = pc.BoxPreconditioner((0, 0, 0, nx, ny, nz), M, H, K0, variant, 0.0)
    two = pc2.TwoLevelBoxPreconditioner((0, 0, 0, nx, ny, nz, 2), M, H, K0, variant)
    np.testing.assert_allclose(two.apply_box(r), one.apply_box(r), atol=1e-13)


def test_blocked_mixed_levels_dense():
    """Block-diagonal preconditioner with a 1-level and a 2-level box
    (Sec. 5.3): each box gets its own inverse, identity elsewhere."""
    nx, ny, nz = 6, 5, 2
    M = _M(nx, ny, nz, 4)
    b1 = (0, 0, 0, 6, 2, 2)
    b2 = (1, 2, 0, 4, 3, 2, 2)
    P = pc.Preconditioner(nx, ny, nz, H, K0, M, [b1, b2], 3, 0.0)
    r = _rng_c(np.random.default_rng(3), 3, nz, ny, nx)
    z = P.apply(r)
    C1 = pc.chan_block_dense(pc.homogenized_box_matrix(b1, M, H, K0, 3), 3 * 2 * 2, 6)
    C2 = pc2.chan2_block_dense(pc2.homogenized_box_matrix2(b2, M, H, K0, 3), 6, 3, 4)
    for b, C in ((b1, C1), (b2, C2)):
        x0, y0, z0, bx, by, bz = b[:6]
        sl = (slice(None), slice(z0, z0 + bz), slice(y0, y0 + by), slice(x0, x0 + bx))
        np.testing.assert_allclose(z[sl].ravel(), np.linalg.solve(C, r[sl].ravel()), atol=1e-12)
    mask = np.ones((3, nz, ny, nx), dtype=bool)
    mask[:, 0:2, 0:2, 0:6] = False
    mask[:, 0:2, 2:5, 1:5] = False
    np.testing.assert_array_equal(z[mask], r[mask])


def test_two_level_preconditioned_gmres_solves_the_system():
    nx, ny, nz = 8, 6, 2
    eps = np.full((nz, ny, nx), inputs.EPS_SIO2, dtype=complex)
    eps[:, 0:5, 1:8] = inputs.EPS_SI          # Si is the modal value, as for a disk box
    eps_bg = inputs.EPS_SIO2
    M = op.material(eps, eps_bg)
    k = op.background_k(K0, eps_bg)
    A = op.dense_matrix(nx, ny, nz, H, k, M)
    b = (M[None] * _rng_c(np.random.default_rng(4), 3, nz, ny, nx))
    P = pc.Preconditioner(nx, ny, nz, H, k, M, [(0, 0, 0, nx, ny, nz, 2)], 1, 0.0)
    res = gmres.gmres(lambda v: (A @ v.ravel()).reshape(v.shape), b, P.apply, tol=1e-12)
    assert res.relres <= 1e-12
    np.testing.assert_allclose(res.x.ravel(), np.linalg.solve(A, b.ravel()), atol=1e-10 * np.abs(b).max())


def test_plane_homogenisation_hand_example():
    """Plane variants of M~ (reading R12) on a 2 x 2 x 3 box written out by hand:
    plane z = 0 holds 1, 1, 1, 1+4j, 0, 0 -> mean (4 + 4j)/6; plane z = 1 is
    all 2 -> mean 2; the mode over the box is 2 (six entries)."""
    M = np.zeros((2, 2, 3), dtype=complex)
    M[0] = [[1, 1, 1], [1 + 4j, 0, 0]]
    M[1] = 2.0
    np.testing.assert_allclose(homogenize.homogenize_plane(M, 2), [(4 + 4j) / 6, 2.0])
    np.testing.assert_allclose(homogenize.homogenize_plane(M, 3), [4 / 6, 2.0])
    np.testing.assert_allclose(homogenize.homogenize_plane(M, 1), [2.0, 2.0])


def test_disk_geometry():
    """Synthetic disk beside a bus (Sec. 5.3.1): the disk covers about pi/4 of
    its box, the bus is one full-length core, the boxes are disjoint and inside
    the grid, the disk box is 2-level, and the disk stays lossless."""
    R = 40
    p = inputs.disk_resonator(R, nz=3, lead=10)
    bus, disk = p.boxes
    assert disk[6] == 2 and len(bus) == 6
    for b in (bus, disk):
        x0, y0, z0, bx, by, bz = b[:6]
        assert x0 >= 0 and y0 >= 0 and x0 + bx <= p.nx and y0 + by <= p.ny and z0 + bz <= p.nz
    assert bus[1] + bus[4] <= disk[1]                          # the gap separates them in y
    x0, y0, _, bx, by, _ = disk[:6]
    core = p.eps[1, y0:y0 + by, x0:x0 + bx].real > 3
    assert abs(core.mean() - math.pi / 4) < 0.02
    assert np.all(p.eps[:, y0:y0 + by, x0:x0 + bx].imag == 0)
    assert np.all(p.eps[1, bus[1]:bus[1] + bus[4], :].real > 3)
