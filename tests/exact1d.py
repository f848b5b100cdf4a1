"""Exact 1D B-spline integrals for pinning the oracle, computed independently of it:
scipy's BSpline/PPoly piecewise polynomials, multiplied coefficient-wise and integrated
in closed form on every breakpoint interval."""
import numpy as np
from scipy.interpolate import BSpline, PPoly


def ppoly_of(U, p, i, deriv=0):
    c = np.zeros(len(U) - p - 1)
    c[i] = 1.0
    b = BSpline(np.asarray(U, float), c, p, extrapolate=False)
    if deriv:
        b = b.derivative(deriv)
    return PPoly.from_spline(b)


def exact_inner(U, p, i, j, deriv=0, a=None, b=None):
    """int_a^b B_i^(deriv) B_j^(deriv) dx exactly (piecewise polynomial product)."""
    P, Q = ppoly_of(U, p, i, deriv), ppoly_of(U, p, j, deriv)
    x = P.x
    assert np.allclose(x, Q.x)
    lo = x[0] if a is None else a
    hi = x[-1] if b is None else b
    tot = 0.0
    for k in range(len(x) - 1):
        l, r = max(x[k], lo), min(x[k + 1], hi)
        if r <= l:
            continue
        # local polynomials in (t - x[k]), highest power first
        pp = np.polymul(P.c[:, k], Q.c[:, k])
        ip = np.polyint(pp)
        tot += np.polyval(ip, r - x[k]) - np.polyval(ip, l - x[k])
    return tot


def cardinal_bspline(m, x):
    """Cardinal B-spline of degree m on [0, m+1] (truncated-power closed form)."""
    from math import comb, factorial
    return sum((-1) ** j * comb(m + 1, j) * max(x - j, 0.0) ** m for j in range(m + 2)) / factorial(m)
