"""Pins for the oracle's system matrix and FFT matvec (Sec. 2, Eq. sys_mat and
the O(n log n) circulant-embedding product of Sec. 1)."""
import itertools
import math

import numpy as np
import pytest

from oracle import greens
from oracle import operator as op
from paper_1903_07884_gb300 import inputs

H = 0.05
K0 = 2 * math.pi / 1.55


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 1), (1, 3, 1), (1, 1, 4), (3, 2, 2),
                                   (5, 3, 2), (4, 4, 3), (2, 5, 3), (5, 1, 5)])
def test_fft_matvec_equals_dense_brute_force(shape):
    nx, ny, nz = shape
    eps = inputs.random_permittivity(nz, ny, nx, seed=nx * 100 + ny * 10 + nz)
    M = op.material(eps, 1.0)
    x = inputs.random_field((3, nz, ny, nx), seed=7)
    A = op.dense_matrix(nx, ny, nz, H, K0, M)
    spec = op.generator_spectra(nx, ny, nz, H, K0)
    y_dense = op.dense_matvec(A, x)
    y_fft = op.fft_matvec(x, M, spec)
    assert np.linalg.norm(y_fft - y_dense) <= 1e-13 * np.linalg.norm(y_dense)


def test_embedding_length_above_minimum_is_exact():
    nx, ny, nz = 5, 3, 2
    M = op.material(inputs.random_permittivity(nz, ny, nx, seed=1), 2.085)
    x = inputs.random_field((3, nz, ny, nx), seed=2)
    k = op.background_k(K0, 2.085)
    y1 = op.fft_matvec(x, M, op.generator_spectra(nx, ny, nz, H, k))
    y2 = op.fft_matvec(x, M, op.generator_spectra(nx, ny, nz, H, k, L=9, Py=7, Pz=3))
    y3 = op.fft_matvec(x, M, op.generator_spectra(nx, ny, nz, H, k, L=16, Py=12, Pz=5))
    assert np.linalg.norm(y2 - y1) <= 1e-13 * np.linalg.norm(y1)
    assert np.linalg.norm(y3 - y1) <= 1e-13 * np.linalg.norm(y1)


def test_N_is_complex_symmetric_and_blocks_have_six_unique():
    nx, ny, nz = 3, 2, 2
    N = nx * ny * nz
    A = op.dense_matrix(nx, ny, nz, H, K0, np.ones((nz, ny, nx)))
    Nmat = np.eye(3 * N) - A          # with M = 1, A = I - N  ->  N = I - A
    np.testing.assert_allclose(Nmat, Nmat.T, atol=1e-15)
    for a, b in itertools.product(range(3), range(3)):
        blk = Nmat[a * N:(a + 1) * N, b * N:(b + 1) * N]
        np.testing.assert_allclose(blk, blk.T, atol=1e-15)   # each block symmetric


def test_single_voxel_closed_form():
    # One voxel: the 3x3 system is diagonal, (1 - M N_ii) w = M e.
    eps = np.array([[[12.11 - 0.3j]]])
    M = op.material(eps, 1.0)[0, 0, 0]
    e = np.array([0.2 + 0.1j, 1.0 - 0.5j, -0.3j]).reshape(3, 1, 1, 1)
    A = op.dense_matrix(1, 1, 1, H, K0, op.material(eps, 1.0))
    w = np.linalg.solve(A, (M * e).ravel())
    Nii = 1.0 + greens.self_term(H, K0)
    np.testing.assert_allclose(w, (M * e.ravel()) / (1 - M * Nii), rtol=1e-14)
    # and N_ii = (2/3)(1 + jka) exp(-jka) for the sphere self term
    a = (3 * H ** 3 / (4 * math.pi)) ** (1 / 3)
    assert abs(Nii - (2 / 3) * (1 + 1j * K0 * a) * np.exp(-1j * K0 * a)) < 1e-15


def test_matrix_row_matches_dense():
    nx, ny, nz = 4, 3, 2
    M = op.material(inputs.random_permittivity(nz, ny, nx, seed=5), 1.0)
    A = op.dense_matrix(nx, ny, nz, H, K0, M)
    for row in (0, 5, 23, 30, 71):
        np.testing.assert_allclose(op.matrix_row(row, nx, ny, nz, H, K0, M), A[row], atol=1e-16)


def test_cladding_rows_are_identity():
    # M = 0 in background voxels: those rows of A are rows of the identity.
    p = inputs.directional_coupler(6, 0.025, 1.55, ny=12, nz=2, core_w=3, gap=2, margin=2)
    M = op.material(p.eps, p.eps_bg)
    k = op.background_k(p.k0, p.eps_bg)
    x = inputs.random_field((3, p.nz, p.ny, p.nx), seed=9)
    y = op.fft_matvec(x, M, op.generator_spectra(p.nx, p.ny, p.nz, p.h, k))
    clad = np.broadcast_to(M == 0, x.shape)
    np.testing.assert_array_equal(y[clad], x[clad])


# --- pins of the material operator, the right-hand side and the background
# wavenumber against values fixed outside the oracle's own formulas ---------

def test_material_recovers_table1_contrasts():
    """Table 1 prints the contrasts the problem is posed with: Si in SiO2 is
    12.1/2.085 ~ 5.80 and Si3N4 in SiO2 is 3.99/2.085 ~ 1.91; materials on
    their own are cladded by air.  M = (eps_r - 1)/eps_r inverts to
    eps_r = 1/(1 - M), which must reproduce those printed contrasts (a missing
    division by the background, or a dropped 1/eps_r, does not)."""
    for eps, eps_bg, printed in ((12.1, 2.085, 5.80), (3.99, 2.085, 1.91), (12.1, 1.0, 12.1),
                                 (2.085, 1.0, 2.085)):
        M = op.material(np.array([[[eps]]], dtype=np.complex128), eps_bg)[0, 0, 0]
        assert abs(1.0 / (1.0 - M) - printed) < 0.006, (eps, eps_bg)
    # the cladding itself is no contrast at all: M = 0, hence b = 0 there
    assert op.material(np.array([[[2.085 + 0j]]]), 2.085)[0, 0, 0] == 0.0


def test_single_voxel_static_limit_is_clausius_mossotti():
    """A lone voxel at k0 -> 0 is a small dielectric sphere (the self term is
    the equal-volume sphere's) in a uniform field.  Electrostatics gives its
    interior field 3 E0 / (eps_r + 2) with eps_r relative to the background,
    and Sec. 2 (j = j omega eps0 (eps_r - 1) e) makes the normalised current
    w = (eps_r - 1) e, so w = 3 (eps_r - 1)/(eps_r + 2) e_inc: the
    Clausius-Mossotti factor.  Pins material, rhs and the system together."""
    eps_bg = 2.085
    eps = np.array([[[12.11 - 0.4j]]])
    e = np.array([0.3 - 0.2j, 1.0 + 0.1j, -0.5j]).reshape(3, 1, 1, 1)
    k = op.background_k(0.0, eps_bg)
    M = op.material(eps, eps_bg)
    A = op.dense_matrix(1, 1, 1, H, k, M)
    w = np.linalg.solve(A, op.rhs(eps, eps_bg, e).ravel())
    er = (12.11 - 0.4j) / eps_bg
    np.testing.assert_allclose(w, 3 * (er - 1) / (er + 2) * e.ravel(), rtol=1e-14)


def test_background_wavenumber_sets_the_wavelength_in_the_cladding():
    """In a background of permittivity eps_b the wavelength is
    lambda_b = lambda0 / sqrt(eps_b).  With voxels of lambda_b / 20, the
    radiating trace sum_a G^{aa}(d) = 2 k^2 V exp(-jkR)/(4 pi R) at R =
    lambda_b and R = 2 lambda_b differ by the factor 1/2 exactly (a whole
    period of phase apart); any other k leaves a phase between them."""
    lam0, eps_bg = 1.55, 2.085
    lam_b = lam0 / math.sqrt(eps_bg)
    h = lam_b / 20
    k = op.background_k(2 * math.pi / lam0, eps_bg)
    G = greens.entries(np.array([20, 40]), np.array([0, 0]), np.array([0, 0]), h, k)
    tr = G[greens.pair_index(0, 0)] + G[greens.pair_index(1, 1)] + G[greens.pair_index(2, 2)]
    ratio = tr[1] / tr[0]
    assert abs(ratio - 0.5) < 1e-12
    # the same voxels in vacuum at the same lambda0 are not a whole period apart
    G0 = greens.entries(np.array([20, 40]), np.array([0, 0]), np.array([0, 0]), h, 2 * math.pi / lam0)
    tr0 = G0[0] + G0[3] + G0[5]
    assert abs(tr0[1] / tr0[0] - 0.5) > 0.1
