"""Pins for the oracle's circulant preconditioner (Sec. 4 Eq. Di and the
C_B^{-1} display, Sec. 5.1.1 Eqs. proxy1-proxy2, Sec. 5.2 homogenisation,
Sec. 5.3 partitioning)."""
import math

import numpy as np
import pytest

from oracle import gmres, homogenize
from oracle import operator as op
from oracle import precond as pc
from paper_1903_07884_gb300 import inputs

H = 0.05
K0 = 2 * math.pi / 1.55


def _box_problem(nx, ny, nz, seed=0, eps_bg=1.0):
    eps = inputs.random_permittivity(nz, ny, nx, seed=seed)
    return op.material(eps, eps_bg)


@pytest.mark.parametrize("shape", [(1, 1, 1), (4, 1, 1), (5, 2, 1), (6, 2, 2), (7, 3, 1), (3, 2, 3)])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_blocks_match_dense_definition(shape, variant):
    """D_f from the closed form (Eq. Chan on generator lines + Eq. Di) equals
    the DFT of the Chan circulants taken from the dense box matrix by their
    Frobenius definition."""
    nx, ny, nz = shape
    M = _box_problem(nx, ny, nz, seed=nx + 7 * ny + 31 * nz)
    bp = pc.BoxPreconditioner((0, 0, 0, nx, ny, nz), M, H, K0, variant, 0.0)
    A = pc.homogenized_box_matrix((0, 0, 0, nx, ny, nz), M, H, K0, variant)
    m = 3 * ny * nz
    C = pc.chan_block_dense(A, m, nx)
    # first column of each circulant block -> eigenvalues -> D_f
    D_def = np.zeros((nx, m, m), dtype=complex)
    for p in range(m):
        for q in range(m):
            col = C[p * nx:(p + 1) * nx, q * nx]
            D_def[:, p, q] = np.fft.fft(col)
    np.testing.assert_allclose(bp.D, D_def, atol=1e-13)


@pytest.mark.parametrize("shape", [(4, 2, 1), (5, 3, 2), (8, 2, 2)])
def test_inverse_of_dense_chan_block(shape):
    """P^{-1}(C_B x) = x with C_B assembled densely from its definition and
    P^{-1} applied through the per-frequency factorisations."""
    nx, ny, nz = shape
    M = _box_problem(nx, ny, nz, seed=3)
    A = pc.homogenized_box_matrix((0, 0, 0, nx, ny, nz), M, H, K0, 3)
    m = 3 * ny * nz
    C = pc.chan_block_dense(A, m, nx)
    P = pc.Preconditioner(nx, ny, nz, H, K0, M, None, 3, 0.0)
    x = inputs.random_field((3, nz, ny, nx), seed=11)
    Cx = (C @ x.ravel()).reshape(x.shape)
    z = P.apply(Cx)
    assert np.linalg.norm(z - x) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("shape", [(6, 2, 2), (7, 3, 2), (10, 1, 3)])
def test_symmetry_S1(shape):
    """D_{n-f} = S D_f S with S = -1 on the x-component rows (x-parity of the
    generators).  Holds to rounding for every homogenisation."""
    nx, ny, nz = shape
    M = _box_problem(nx, ny, nz, seed=4)
    bp = pc.BoxPreconditioner((0, 0, 0, nx, ny, nz), M, H, K0, 2, 0.0)
    a, _, _ = pc.box_order(ny, nz)
    S = np.where(a == 0, -1.0, 1.0)
    for f in range(1, nx):
        np.testing.assert_allclose(bp.D[nx - f], S[:, None] * bp.D[f] * S[None, :], atol=1e-13)


def test_reduction_tau_zero_keeps_all_and_kept_blocks_identical():
    n = 41
    p = inputs.straight_guide(n, 8, 4, 0.05, 1.55, absorber=4)
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    full = pc.BoxPreconditioner((0, 0, 0, n, 8, 4), M, p.h, k, 3, 0.0)
    assert len(full.kept) == n
    red = pc.BoxPreconditioner((0, 0, 0, n, 8, 4), M, p.h, k, 3, 1e-3)
    assert 0 < len(red.kept) < n
    for f in red.kept:
        np.testing.assert_array_equal(red.D[f], full.D[f])
    # discarded frequencies use the central block D_{ceil(n/2)} (1-based)
    assert red.rep == 20
    f_disc = [f for f in range(n) if not red.keep_mask[f]]
    assert f_disc and all(red.block_for(f) == 20 for f in f_disc)
    # the kept set is symmetric under f -> n - f (x-parity of the proxy entry)
    ks = set(int(f) for f in red.kept)
    assert all(((n - f) % n) in ks for f in ks)
    # low |frequency| blocks are the distinct ones (Fig. abs(a))
    assert 0 in ks and 1 in ks


def test_proxy_definition_hand_case():
    """v^ = |v| / ||v||_inf with v_f the (1, c*) entry, c* = ceil(ny/2) ceil(nz/2)
    (1-based); for ny = 6, nz = 4 that is 3 * 2 = 6, i.e. 0-based column 5 =
    (alpha x, z 0, y 5).  Checked against D_f itself when M~_0 != 0."""
    nx, ny, nz = 12, 6, 4
    M = np.full((nz, ny, nx), 0.9 + 0.0j)
    bp = pc.BoxPreconditioner((0, 0, 0, nx, ny, nz), M, H, K0, 3, 1e-3)
    v = bp.D[:, 0, 5]
    ref = np.abs(v) / np.abs(v).max()
    np.testing.assert_allclose(bp.vhat, ref, rtol=1e-12)


def test_partition_identity_outside_boxes_and_single_box():
    nx, ny, nz = 10, 6, 2
    M = _box_problem(nx, ny, nz, seed=8)
    x = inputs.random_field((3, nz, ny, nx), seed=12)
    boxes = [(0, 0, 0, 10, 2, 2), (1, 3, 0, 7, 3, 2)]
    P = pc.Preconditioner(nx, ny, nz, H, K0, M, boxes, 3, 0.0)
    z = P.apply(x)
    inside = np.zeros((nz, ny, nx), dtype=bool)
    for (x0, y0, z0, a, b, c) in boxes:
        inside[z0:z0 + c, y0:y0 + b, x0:x0 + a] = True
    out = np.broadcast_to(~inside, x.shape)
    np.testing.assert_array_equal(z[out], x[out])
    # each box block equals a standalone preconditioner on that box's data
    for bx in boxes:
        x0, y0, z0, a, b, c = bx
        sl = (slice(None), slice(z0, z0 + c), slice(y0, y0 + b), slice(x0, x0 + a))
        sub = pc.Preconditioner(a, b, c, H, K0, np.ascontiguousarray(M[sl[1:]]), None, 3, 0.0)
        np.testing.assert_allclose(z[sl], sub.apply(np.ascontiguousarray(x[sl])), atol=1e-13)
    # one whole-grid box is the unpartitioned preconditioner
    P1 = pc.Preconditioner(nx, ny, nz, H, K0, M, [(0, 0, 0, nx, ny, nz)], 3, 0.0)
    P0 = pc.Preconditioner(nx, ny, nz, H, K0, M, None, 3, 0.0)
    np.testing.assert_array_equal(P1.apply(x), P0.apply(x))


def test_exact_preconditioner_converges_in_one_step():
    """If the operator is its own circulant-block approximation (x-periodic
    structure, homogeneous M), the preconditioner is exact and right-
    preconditioned GMRES converges in one iteration."""
    nx, ny, nz = 8, 3, 2
    M = np.full((nz, ny, nx), 0.7 - 0.05j)
    A = pc.homogenized_box_matrix((0, 0, 0, nx, ny, nz), M, H, K0, 2)
    C = pc.chan_block_dense(A, 3 * ny * nz, nx)
    P = pc.Preconditioner(nx, ny, nz, H, K0, M, None, 2, 0.0)
    b = inputs.random_field((3, nz, ny, nx), seed=2)
    res = gmres.gmres(lambda v: (C @ v.ravel()).reshape(v.shape), b, P.apply, tol=1e-12)
    assert res.iters == 1 and res.relres < 1e-12
