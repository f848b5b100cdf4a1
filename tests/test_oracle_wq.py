"""Pins for the oracle's WQ and DWQ rules (Sec. 1 WQ ingredient; Sec. 2.2 steps 1-6 and
the Gauss-superset paragraph).  Exact integrals come from scipy piecewise polynomials
(tests/exact1d.py), not from the oracle."""
import numpy as np
import pytest
from scipy.linalg import null_space

from oracle.wq import Space1D
from oracle.bspline import basis_all
from tests.exact1d import exact_inner

CASES = [(8, 2), (9, 3), (10, 4), (12, 5), (14, 6), (3, 3), (2, 4)]


def _check_rule(sp, U, i, Q, wQ, kind, a=None, b=None, tol=1e-13):
    p = sp.p
    N, dN = basis_all(U, p, sp.t_sup[Q])
    F = N if kind == "00" else dN
    der = 0 if kind == "00" else 1
    n = len(U) - p - 1
    res = []
    for j in range(n):
        lhs = np.dot(wQ, F[j])
        rhs = exact_inner(U, p, i, j, der, a, b)
        res.append((lhs, rhs))
    res = np.array(res)
    scale = max(np.max(np.abs(res[:, 1])), 1e-300)
    assert np.max(np.abs(res[:, 0] - res[:, 1])) <= tol * scale, np.max(np.abs(res[:, 0] - res[:, 1])) / scale


@pytest.mark.parametrize("n_el,p", CASES)
@pytest.mark.parametrize("kind", ["00", "11"])
def test_standard_rule_exactness(n_el, p, kind):
    """sum_q w_i(q) B_j(t_q) = int B_i B_j for every trial function j (and the w11 analogue)."""
    sp = Space1D(n_el, p)
    for i in range(sp.n):
        Q, wQ = sp.std_rule(i, kind)
        _check_rule(sp, sp.U, i, Q, wQ, kind, tol=5e-13 if p >= 5 else 1e-13)


@pytest.mark.parametrize("n_el,p", CASES)
def test_standard_rule_layout_and_minnorm(n_el, p):
    sp = Space1D(n_el, p)
    if n_el >= 2:
        assert len(sp.wq_idx) == 2 * (p + 1) + 2 * (n_el - 2)
    N, dN = basis_all(sp.U, p, sp.t_sup)
    for kind, F in (("00", N), ("11", dN)):
        for i in range(sp.n):
            Q, wQ = sp.std_rule(i, kind)
            e_lo, e_hi = sp.supp_elems(i)
            assert set(sp.elem_of_sup[Q]) == set(range(e_lo, e_hi + 1))
            assert np.all(sp.wq_mask[Q])
            J = [j for j in range(sp.n) if abs(j - i) <= p]
            A = F[np.ix_(J, Q)]
            full = all(np.all(sp.wq_mask[sp.elem_of_sup == e]) for e in range(e_lo, e_hi + 1))
            if full:  # Gauss shortcut: w = g * B_i
                assert np.allclose(wQ, sp.w_sup[Q] * F[i, Q], rtol=0, atol=1e-16)
            else:     # minimum norm: w lies in the row space of A (orthogonal to null(A))
                Z = null_space(A)
                if Z.size:
                    assert np.linalg.norm(Z.T @ wQ) <= 1e-9 * np.linalg.norm(wQ)


@pytest.mark.parametrize("n_el,p", [(8, 2), (9, 3), (10, 4), (12, 5), (14, 6)])
@pytest.mark.parametrize("kind", ["00", "11"])
def test_dwq_one_sided_exactness(n_el, p, kind):
    """The one-sided DWQ rule integrates B_i B_j exactly over the kept side of the
    artificial discontinuity, for every original trial function j, and is zero on the
    far side (Sec. 2.2 steps 3-6 and the one-sidedness remark)."""
    sp = Space1D(n_el, p)
    for i in range(sp.n):
        e_lo, e_hi = sp.supp_elems(i)
        for b in sp.dwq_candidates(i):
            for side in (0, 1):
                w = sp.dwq_rule(i, b, side, kind)
                kept = range(e_lo, b) if side == 0 else range(b, e_hi + 1)
                assert np.all(w[~np.isin(sp.elem_of_sup, list(kept))] == 0.0)
                a_, b_ = (sp.xb[e_lo], sp.xb[b]) if side == 0 else (sp.xb[b], sp.xb[e_hi + 1])
                Q = np.nonzero(w)[0]
                _check_rule(sp, sp.U, i, Q, w[Q], kind, a_, b_, tol=2e-12 if p >= 5 else 1e-13)


@pytest.mark.parametrize("n_el,p", [(8, 2), (9, 3), (10, 4), (12, 6)])
def test_dwq_gauss_shortcut_identity(n_el, p):
    """When every kept element carries the full Gauss set, the knot-insertion DWQ rule
    equals the Gauss-folded rule g_q B_i(t_q) (Sec. 2.2, last paragraph)."""
    sp = Space1D(n_el, p)
    N, dN = basis_all(sp.U, p, sp.t_sup)
    hits = 0
    for i in range(sp.n):
        e_lo, e_hi = sp.supp_elems(i)
        for b in sp.dwq_candidates(i):
            for side in (0, 1):
                kept = list(range(e_lo, b)) if side == 0 else list(range(b, e_hi + 1))
                layout = sp.wq_mask | (sp.elem_of_sup == b - 1) | (sp.elem_of_sup == b)
                if not all(np.all(layout[sp.elem_of_sup == e]) for e in kept):
                    continue
                hits += 1
                for kind, F in (("00", N), ("11", dN)):
                    w_short = sp.dwq_rule(i, b, side, kind)
                    w_ref = sp.dwq_rule(i, b, side, kind, force_refined=True)
                    sel = np.isin(sp.elem_of_sup, kept)
                    assert np.allclose(w_short[sel], sp.w_sup[sel] * F[i, sel], rtol=0, atol=1e-16)
                    assert np.max(np.abs(w_short - w_ref)) <= 1e-12 * np.max(np.abs(w_short))
    assert hits > 0
