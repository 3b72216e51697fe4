"""Pins for the oracle's Green's-tensor generator entries (reading of Eq. op_N,
Sec. 2).  Each check comes from mathematics independent of the oracle code:
symbolic differentiation of g, quadrature, the static dipole field, the trace
identity of the Helmholtz equation, far-field transversality and radiation
reaction."""
import math

import numpy as np
import pytest
import sympy as sp
from scipy import integrate

from oracle import greens

H = 0.05
K = 2 * math.pi / 1.55


def _symbolic_kernel():
    x, y, z, k = sp.symbols("x y z k", real=True)
    R = sp.sqrt(x * x + y * y + z * z)
    g = sp.exp(-sp.I * k * R) / (4 * sp.pi * R)
    X = (x, y, z)
    out = {}
    for i, (a, b) in enumerate(greens.PAIRS):
        expr = sp.diff(g, X[a], X[b]) + (k * k * g if a == b else 0)
        out[i] = sp.lambdify((x, y, z, k), expr, "mpmath")
    return out


@pytest.fixture(scope="module")
def sym_kernel():
    return _symbolic_kernel()


@pytest.mark.parametrize("d", [(1, 0, 0), (0, 1, 0), (1, 1, 0), (2, -1, 3), (-3, 2, -1), (7, 0, -2), (1, 2, 3)])
@pytest.mark.parametrize("k", [K, 3.48 * K, 0.3])
def test_offdiagonal_equals_symbolic_second_derivative(sym_kernel, d, k):
    import mpmath
    mpmath.mp.dps = 30
    G = greens.entries(*d, H, k)
    V = H ** 3
    for i in range(6):
        ref = complex(sym_kernel[i](d[0] * H, d[1] * H, d[2] * H, k)) * V
        assert abs(G[i] - ref) <= 1e-12 * max(abs(ref), 1e-3 * abs(G).max())


def test_static_limit_is_dipole_field():
    d = np.array([2, -1, 3])
    R = H * np.linalg.norm(d)
    r = d / np.linalg.norm(d)
    G = greens.entries(*d, H, 0.0)
    V = H ** 3
    for i, (a, b) in enumerate(greens.PAIRS):
        ref = V * (3 * r[a] * r[b] - (a == b)) / (4 * math.pi * R ** 3)
        assert abs(G[i] - ref) < 1e-14


def test_trace_identity():
    rng = np.random.default_rng(3)
    d = rng.integers(-6, 7, size=(3, 50))
    d = d[:, np.any(d != 0, axis=0)]
    G = greens.entries(d[0], d[1], d[2], H, K)
    R = H * np.sqrt((d ** 2).sum(0))
    g = np.exp(-1j * K * R) / (4 * math.pi * R)
    tr = G[greens.pair_index(0, 0)] + G[greens.pair_index(1, 1)] + G[greens.pair_index(2, 2)]
    np.testing.assert_allclose(tr, 2 * K * K * H ** 3 * g, rtol=1e-12)


def test_far_field_is_transverse():
    d = np.array([400, 300, 0])          # kR ~ 100; near-field terms are O(1/(kR))
    R = H * np.linalg.norm(d)
    r = d / np.linalg.norm(d)
    G = greens.entries(*d, H, K)
    g = np.exp(-1j * K * R) / (4 * math.pi * R)
    for i, (a, b) in enumerate(greens.PAIRS):
        ref = H ** 3 * K * K * g * ((a == b) - r[a] * r[b])
        assert abs(G[i] - ref) < (2.0 / (K * R)) * abs(H ** 3 * K * K * g)


def test_parity_and_reciprocity():
    rng = np.random.default_rng(4)
    for _ in range(20):
        d = rng.integers(-5, 6, size=3)
        if not d.any():
            continue
        G = greens.entries(*d, H, K)
        Gm = greens.entries(*(-d), H, K)
        np.testing.assert_allclose(G, Gm, rtol=1e-14, atol=0)     # G(d) = G(-d)
        for axis in range(3):
            dd = d.copy(); dd[axis] = -dd[axis]
            Gf = greens.entries(*dd, H, K)
            for i, (a, b) in enumerate(greens.PAIRS):
                assert abs(Gf[i] - greens.parity(a, b, axis) * G[i]) <= 1e-14 * abs(G).max()


def test_self_term_static_depolarisation():
    assert abs(greens.self_term(H, 0.0) - (-1.0 / 3.0)) < 1e-15


def test_self_term_matches_quadrature():
    # G_self = -1/3 + (2/3) k^2 int_0^a r exp(-jkr) dr  (field at the centre of
    # a uniformly polarised sphere); the radial integral by quadrature.
    for k in (K, 3.48 * K, 20.0):
        a = (3 * H ** 3 / (4 * math.pi)) ** (1 / 3)
        re = integrate.quad(lambda r: r * math.cos(k * r), 0, a, epsabs=1e-18, epsrel=1e-13)[0]
        im = integrate.quad(lambda r: -r * math.sin(k * r), 0, a, epsabs=1e-18, epsrel=1e-13)[0]
        ref = -1 / 3 + (2 / 3) * k * k * (re + 1j * im)
        assert abs(greens.self_term(H, k) - ref) < 1e-13


def test_self_term_radiation_reaction():
    # Small sphere: Im part is the dipole radiation reaction -(2/9)(ka)^3 and
    # the real part -1/3 + (ka)^2/3.
    for k in (0.5, 1.0, 2.0):
        a = (3 * H ** 3 / (4 * math.pi)) ** (1 / 3)
        ka = k * a
        st = greens.self_term(H, k)
        assert abs(st.imag - (-(2 / 9) * ka ** 3)) < 1e-3 * (2 / 9) * ka ** 3 + 1e-16
        assert abs(st.real - (-1 / 3 + ka * ka / 3)) < 1e-2 * ka * ka
