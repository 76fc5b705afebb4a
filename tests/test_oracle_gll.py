"""Pins for the oracle's GLL nodes, weights and derivative matrix (CPU only).

Each check is independent of the oracle's own formulas: textbook closed forms
(tests/golden), numpy's Legendre roots, quadrature exactness and exact
differentiation of polynomials.
"""
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _closed_forms():
    rows = {}
    for line in open(os.path.join(GOLD, "gll_closed_forms.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        n, x, w = (s.strip() for s in line.split("|"))
        env = {"sqrt": math.sqrt}
        rows.setdefault(int(n), []).append((eval(x, env), eval(w, env)))
    return rows


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_gll_closed_forms(orc, N):
    xs, ws = zip(*_closed_forms()[N])
    xi, w = orc.gll(N)
    np.testing.assert_allclose(xi, xs, atol=1e-15)
    np.testing.assert_allclose(w, ws, rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_vs_numpy_legendre(orc, N):
    xi, w = orc.gll(N)
    inner = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real) if N > 1 else []
    np.testing.assert_allclose(xi[1:-1], inner, atol=1e-13)
    assert xi[0] == -1.0 and xi[-1] == 1.0
    assert abs(w.sum() - 2.0) < 1e-13


@pytest.mark.parametrize("N", [2, 4, 7, 9])
def test_gll_quadrature_exact(orc, N):
    # Lobatto quadrature is exact for polynomials of degree <= 2N-1
    xi, w = orc.gll(N)
    for p in range(2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(w @ xi ** p - exact) < 1e-13


def test_dmat_n2_golden(orc):
    ref = np.loadtxt(os.path.join(GOLD, "dmat_n2.txt"))
    np.testing.assert_allclose(orc.dmat(2), ref, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_dmat_exact_on_polynomials(orc, N):
    xi, _ = orc.gll(N)
    D = orc.dmat(N)
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-12
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-12
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-11 * N * N)
    for p in range(1, N + 1):
        np.testing.assert_allclose(D @ xi ** p, p * xi ** (p - 1), atol=2e-12 * N * N)


def test_dmat_n7_value(orc):
    assert orc.dmat(7)[0, 0] == -14.0
