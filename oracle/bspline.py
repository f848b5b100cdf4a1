"""Oracle 1D spline toolkit (test infrastructure only; see ``oracle/__init__``).

Gauss-Legendre rules, open knot vectors, Cox-de Boor values and first
derivatives, and knot insertion.  These are the univariate ingredients of the
paper's method: the Gauss superset of Sec. 2.2 (last paragraph), the B-spline
background mesh of Sec. 1 and the knot insertion with subdivision matrix S of
Sec. 2.2 step 3.  Written from the textbook definitions, deliberately plain.
"""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes/weights on [-1, 1], ascending.

    Newton's method on P_n, with P_n evaluated by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and
    P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weights 2 / ((1-x^2) P_n'^2).
    """
    if n < 1:
        raise ValueError("n >= 1")
    xs, ws = [], []
    for i in range(n):
        z = np.cos(np.pi * (i + 0.75) / (n + 0.5))
        for _ in range(100):
            pkm1, pk = 1.0, z
            for k in range(1, n):
                pkm1, pk = pk, ((2 * k + 1) * z * pk - k * pkm1) / (k + 1)
            dp = n * (z * pk - pkm1) / (z * z - 1.0)
            dz = pk / dp
            z -= dz
            if abs(dz) < 1e-15:
                break
        pkm1, pk = 1.0, z
        for k in range(1, n):
            pkm1, pk = pk, ((2 * k + 1) * z * pk - k * pkm1) / (k + 1)
        dp = n * (z * pk - pkm1) / (z * z - 1.0)
        xs.append(z)
        ws.append(2.0 / ((1.0 - z * z) * dp * dp))
    order = np.argsort(xs)
    return np.asarray(xs)[order], np.asarray(ws)[order]


def open_knots(n_el, p, lo=0.0, hi=1.0):
    """Open uniform knot vector [lo^{p+1}, interior..., hi^{p+1}].

    Interior knot k (1 <= k < n_el) has the value lo + (hi - lo) * (k / n_el).
    n = n_el + p basis functions; element e spans knots U[e+p], U[e+p+1].
    """
    inner = [lo + (hi - lo) * (k / n_el) for k in range(1, n_el)]
    return np.array([lo] * (p + 1) + inner + [hi] * (p + 1), dtype=np.float64)


def element_bounds(n_el, lo=0.0, hi=1.0):
    """Breakpoints x_0 = lo < x_1 < ... < x_{n_el} = hi (same formula as the knots)."""
    return np.array([lo] + [lo + (hi - lo) * (k / n_el) for k in range(1, n_el)] + [hi],
                    dtype=np.float64)


def _div(a, b):
    """a / b with the Cox-de Boor convention 0/0 := 0 (zero-length spans)."""
    out = np.zeros(np.broadcast(a, b).shape)
    nz = b != 0
    np.divide(a, b, out=out, where=nz)
    return out


def basis_all(U, p, x):
    """All B-splines of degree p on knot vector U at points x.

    Returns (N, dN), each of shape (len(U) - p - 1, len(x)): N[i, k] = B_{i,p}(x_k)
    and dN[i, k] = B'_{i,p}(x_k).  Direct Cox-de Boor recurrence

        B_{i,0}(x) = 1 if U_i <= x < U_{i+1} else 0,
        B_{i,q}(x) = (x - U_i)/(U_{i+q} - U_i) B_{i,q-1}(x)
                   + (U_{i+q+1} - x)/(U_{i+q+1} - U_{i+1}) B_{i+1,q-1}(x),
        B'_{i,p}(x) = p/(U_{i+p} - U_i) B_{i,p-1}(x) - p/(U_{i+p+1} - U_{i+1}) B_{i+1,p-1}(x),

    with 0/0 = 0.  The right end x = U[-1] is assigned to the last non-empty span.
    """
    U = np.asarray(U, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(U) - 1
    lo_, hi_ = U[:-1, None], U[1:, None]
    N = ((lo_ <= x[None, :]) & (x[None, :] < hi_)).astype(np.float64)
    at_end = x == U[-1]
    if np.any(at_end):
        last = max(k for k in range(m) if U[k] < U[k + 1])
        N[last, at_end] = 1.0
    Nprev = N
    for q in range(1, p + 1):
        cnt = m - q
        Ui = U[:cnt, None]
        Uiq = U[q:q + cnt, None]
        Ui1 = U[1:1 + cnt, None]
        Uiq1 = U[q + 1:q + 1 + cnt, None]
        a = _div(x[None, :] - Ui, np.broadcast_to(Uiq - Ui, (cnt, len(x))))
        b = _div(Uiq1 - x[None, :], np.broadcast_to(Uiq1 - Ui1, (cnt, len(x))))
        Nq = a * Nprev[:cnt] + b * Nprev[1:cnt + 1]
        if q == p:
            # derivative uses the degree p-1 functions
            if p == 0:
                dN = np.zeros_like(Nq)
            else:
                c1 = _div(np.full((cnt, 1), float(p)), Uiq - Ui)
                c2 = _div(np.full((cnt, 1), float(p)), Uiq1 - Ui1)
                dN = c1 * Nprev[:cnt] - c2 * Nprev[1:cnt + 1]
        Nprev = Nq
    if p == 0:
        return Nprev, np.zeros_like(Nprev)
    return Nprev, dN


def basis_local(U, p, span, x):
    """The p+1 functions B_{span-p..span} at points x in [U_span, U_{span+1}).

    Same recurrence as ``basis_all``, applied to the 2p+2 knots U[span-p .. span+p+1]
    on which those functions depend.  Returns (N, dN) of shape (p+1, len(x)).
    """
    U = np.asarray(U, dtype=np.float64)
    return basis_all(U[span - p:span + p + 2], p, x)


def insert_knot_matrix(U, p, xi):
    """Insert xi once.  Returns (U_new, T) with coefficients d = T c, i.e.
    sum_i c_i B_i = sum_k d_k Btilde_k, so B_i = sum_k T[k, i] Btilde_k.

    Boehm's rule: with span s (U_s <= xi < U_{s+1}) and
    alpha_k = (xi - U_k) / (U_{k+p} - U_k):  d_k = c_k (k <= s-p),
    d_k = alpha_k c_k + (1 - alpha_k) c_{k-1} (s-p+1 <= k <= s), d_k = c_{k-1} (k > s).
    """
    U = np.asarray(U, dtype=np.float64)
    n = len(U) - p - 1
    s = int(np.searchsorted(U, xi, side="right") - 1)
    T = np.zeros((n + 1, n))
    for k in range(n + 1):
        if k <= s - p:
            T[k, k] = 1.0
        elif k <= s:
            alpha = (xi - U[k]) / (U[k + p] - U[k])
            T[k, k] = alpha
            T[k, k - 1] = 1.0 - alpha
        else:
            T[k, k - 1] = 1.0
    U_new = np.concatenate([U[:s + 1], [xi], U[s + 1:]])
    return U_new, T


def subdivision_matrix(U, p, xi, times):
    """Insert xi `times` times (Sec. 2.2 step 3).  Returns (U_ref, S) with
    S[i, k] the coefficient of refined function k in original function i:
    B_i = sum_k S[i, k] Btilde_k."""
    Ucur = np.asarray(U, dtype=np.float64)
    Ttot = np.eye(len(Ucur) - p - 1)
    for _ in range(times):
        Ucur, T = insert_knot_matrix(Ucur, p, xi)
        Ttot = T @ Ttot
    return Ucur, Ttot.T
