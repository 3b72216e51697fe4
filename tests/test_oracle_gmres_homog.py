"""Pins for the oracle GMRES and homogenisation (Sec. 5.2)."""
import math

import numpy as np
import pytest

from oracle import gmres, homogenize, solve
from oracle import operator as op
from oracle import precond as pc
from paper_1903_07884_gb300 import inputs


def test_gmres_matches_direct_solve_random():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3 + 1j * rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x_ref = np.linalg.solve(A, b)
    for restart in (5, 50):
        r = gmres.gmres(lambda v: A @ v, b, tol=1e-13, restart=restart, max_iter=2000)
        assert r.converged
        assert np.linalg.norm(r.x - x_ref) <= 1e-11 * np.linalg.norm(x_ref)
    # right preconditioning with the exact inverse: one iteration
    Ainv = np.linalg.inv(A)
    r = gmres.gmres(lambda v: A @ v, b, lambda v: Ainv @ v, tol=1e-12)
    assert r.iters == 1


def test_givens_zeroes_second_entry():
    for a, b in [(1 + 2j, 3 - 1j), (0.0, 2j), (1j, 0.0), (-3.0, 4.0)]:
        c, s = gmres.givens(a, b)
        assert abs(-np.conj(s) * a + c * b) < 1e-15
        assert abs(abs(c * a + s * b) - math.hypot(abs(a), abs(b))) < 1e-14


def test_gmres_vie_matches_dense_lu():
    p = inputs.straight_guide(16, 4, 2, 0.05, 1.55, absorber=3)
    x_ref = solve.dense_solve(p)
    s = solve.iterative_solve(p, tol=1e-13, tau=0.0)
    assert np.linalg.norm(s.w - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


@pytest.mark.slow
def test_gmres_small_straight_workload_matches_dense_lu():
    p = inputs.workload_small_straight()
    x_ref = solve.dense_solve(p)
    s = solve.iterative_solve(p, tol=1e-12, tau=1e-3)
    assert np.linalg.norm(s.w - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_homogenisation_hand_example():
    # M over a 1 x 1 x 4 box: values along x
    vals = np.array([0.5 + 0.1j, 0.5 + 0.1j, 0.9 - 0.2j, 0.1 + 0.0j]).reshape(1, 1, 4)
    assert homogenize.homogenize(vals, 1)[0, 0] == 0.5 + 0.1j               # mode
    np.testing.assert_allclose(homogenize.homogenize(vals, 2)[0, 0], (2.0 + 0.0j) / 4)  # mean
    np.testing.assert_allclose(homogenize.homogenize(vals, 3)[0, 0], 0.5)    # real part of the mean
    # mode tie broken by the smallest |value|
    tie = np.array([0.9, 0.9, 0.2, 0.2]).reshape(1, 1, 4).astype(complex)
    assert homogenize.homogenize(tie, 1)[0, 0] == 0.2


def test_homogenised_straight_guide_is_exact_without_absorbers():
    # uniform guide without absorbers: every variant returns M itself
    p = inputs.straight_guide(12, 3, 2, 0.05, 1.55, absorber=0)
    M = op.material(p.eps, p.eps_bg)
    for v in (1, 2, 3):
        np.testing.assert_allclose(homogenize.homogenize(M, v), M[:, :, 0], atol=1e-15)


def test_preconditioned_iterations_flat_in_length():
    """Qualitative regression of Sec. 5.1: with the 1-level preconditioner the
    iteration count of a uniform guide barely grows with its length."""
    its = []
    for nx in (32, 128):
        p = inputs.straight_guide(nx, 4, 2, 0.05, 1.55, absorber=0)
        s = solve.iterative_solve(p, tol=1e-6, tau=0.0)
        its.append(s.iters)
    assert its[1] <= its[0] + 3
