"""Pins for the oracle's 1D toolkit against numpy/scipy library routines, closed forms
and invariants (nothing here compares the oracle with itself)."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import gauss_legendre, open_knots, basis_all, basis_local, subdivision_matrix
from tests.exact1d import cardinal_bspline


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_matches_numpy_leggauss(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-15
    assert np.max(np.abs(w - wr)) < 1e-15


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_monomial_exactness(n):
    x, w = gauss_legendre(n)
    assert abs(w.sum() - 2.0) < 1e-15
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 2e-15


def test_gauss_closed_forms():
    x, w = gauss_legendre(1)
    assert x[0] == 0.0 and w[0] == 2.0
    x, w = gauss_legendre(2)
    assert np.allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15, rtol=0)
    assert np.allclose(w, [1, 1], atol=1e-15, rtol=0)
    x, w = gauss_legendre(3)
    assert np.allclose(x, [-np.sqrt(0.6), 0, np.sqrt(0.6)], atol=1e-15, rtol=0)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15, rtol=0)


def _knot_vectors():
    yield open_knots(7, 2), 2
    yield open_knots(9, 4, -1.0, 1.0), 4
    yield open_knots(5, 6), 6
    rng = np.random.default_rng(11)
    inner = np.sort(rng.uniform(0.1, 0.9, 6))
    U = np.concatenate([[0.0] * 4, inner[:3], [inner[3]] * 2, inner[4:], [1.0] * 4])  # a double knot
    yield U, 3


@pytest.mark.parametrize("case", list(range(4)))
def test_cox_de_boor_matches_scipy(case):
    U, p = list(_knot_vectors())[case]
    rng = np.random.default_rng(case)
    x = rng.uniform(U[0], U[-1], 200)
    N, dN = basis_all(U, p, x)
    n = len(U) - p - 1
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        b = BSpline(U, c, p)
        assert np.max(np.abs(N[i] - b(x))) < 1e-14
        assert np.max(np.abs(dN[i] - b.derivative()(x))) < 1e-11 * max(1.0, np.max(np.abs(dN[i])))
    assert np.max(np.abs(N.sum(axis=0) - 1.0)) < 1e-14       # partition of unity
    assert np.max(np.abs(dN.sum(axis=0))) < 1e-11            # derivatives of a constant


def test_uniform_quadratic_closed_form():
    # interior uniform quadratic: pieces t^2/2, (-2t^2+6t-3)/2, (3-t)^2/2 on [0,1],[1,2],[2,3]
    U = open_knots(10, 2)
    h = 0.1
    i = 5  # support [U_5, U_8] = [0.3, 0.6]
    t = np.linspace(0, 3, 301)[1:-1]
    x = U[i] + h * t
    ref = np.where(t < 1, t ** 2 / 2, np.where(t < 2, (-2 * t ** 2 + 6 * t - 3) / 2, (3 - t) ** 2 / 2))
    N, _ = basis_all(U, 2, x)
    assert np.max(np.abs(N[i] - ref)) < 1e-14
    # the cardinal B-spline formula agrees as well
    assert np.max(np.abs(ref - np.array([cardinal_bspline(2, v) for v in t]))) < 1e-14


def test_basis_local_equals_rows_of_basis_all():
    U, p = open_knots(8, 3), 3
    for e in range(8):
        x = np.linspace(U[e + p], U[e + p + 1], 9)[1:-1]
        N, dN = basis_all(U, p, x)
        Nl, dNl = basis_local(U, p, e + p, x)
        assert np.array_equal(N[e:e + p + 1], Nl)
        assert np.array_equal(dN[e:e + p + 1], dNl)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_knot_insertion_identity(p):
    """B_i = sum_k S_ik Btilde_k after inserting an interior knot p times (C^{-1})."""
    U = open_knots(9, p)
    xi = U[p + 4]
    Ur, S = subdivision_matrix(U, p, xi, p)
    assert np.sum(Ur == xi) == p + 1
    x = np.random.default_rng(p).uniform(0, 1, 100)
    N, _ = basis_all(U, p, x)
    Nr, _ = basis_all(Ur, p, x)
    assert np.max(np.abs(N - S @ Nr)) < 1e-14
    # every original function splits into exactly p+1 refined functions with positive weights
    nz = (S > 0).sum(axis=1)
    for i in range(len(U) - p - 1):
        lo, hi = U[i], U[i + p + 1]
        expect = p + 1 if lo < xi < hi else 1
        assert nz[i] == expect
