"""Pins for T. Chan's optimal circulant and its diagonalisation (Sec. 4,
Eq. Chan)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import circulant

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chan_hand_example.json")


def test_hand_worked_example():
    d = json.load(open(GOLDEN))
    n = d["n"]
    t = {int(k): v for k, v in d["t"].items()}
    t_pos = np.array([t[i] for i in range(n)], dtype=float)
    t_neg = np.array([0.0] + [t[-i] for i in range(1, n)])
    c = circulant.chan_closed_form(t_pos, t_neg)
    ref = np.array([float(Fraction(s)) for s in d["c"]])
    np.testing.assert_allclose(c.real, ref, rtol=0, atol=1e-15)
    # definition route (wrapped-diagonal mean of the Toeplitz matrix)
    c_def = circulant.chan_from_matrix(circulant.toeplitz(t_pos, t_neg))
    np.testing.assert_allclose(c_def.real, ref, atol=1e-15)
    lam = circulant.eigenvalues(c)
    ev = d["circulant_eigenvalues"]
    for f in range(3):
        re, im = ev[f"lambda_{f}"]
        assert abs(lam[f] - (re + 1j * im)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33])
def test_closed_form_equals_frobenius_definition(n):
    rng = np.random.default_rng(n)
    t_pos = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    t_neg = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    t_neg[0] = t_pos[0]
    T = circulant.toeplitz(t_pos, t_neg)
    c_closed = circulant.chan_closed_form(t_pos, t_neg)
    c_def = circulant.chan_from_matrix(T)
    np.testing.assert_allclose(c_closed, c_def, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("n", [4, 9])
def test_frobenius_optimality(n):
    rng = np.random.default_rng(10 + n)
    T = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))   # any matrix
    C = circulant.circulant(circulant.chan_from_matrix(T))
    base = np.linalg.norm(C - T)
    # stationarity: C - T is orthogonal to every circulant basis matrix E_k
    for k in range(n):
        E = circulant.circulant(np.eye(n)[k])
        assert abs(np.vdot(E, C - T)) < 1e-12
    # and any circulant perturbation increases the distance
    for _ in range(20):
        d = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        assert np.linalg.norm(C + 1e-3 * circulant.circulant(d) - T) > base


def test_circulant_is_its_own_chan():
    rng = np.random.default_rng(1)
    c = rng.standard_normal(11) + 1j * rng.standard_normal(11)
    C = circulant.circulant(c)
    np.testing.assert_allclose(circulant.chan_from_matrix(C), c, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_diagonalisation(n):
    rng = np.random.default_rng(20 + n)
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    C = circulant.circulant(c)
    lam = circulant.eigenvalues(c)
    ev = np.linalg.eigvals(C)
    # same multiset of eigenvalues
    for l in lam:
        assert np.min(np.abs(ev - l)) < 1e-10 * max(1, abs(l))
    F = circulant.dft_matrix(n)
    np.testing.assert_allclose(np.linalg.inv(F) @ np.diag(lam) @ F, C, atol=1e-12)
