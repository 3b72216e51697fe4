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
