"""Pins for the oracle's O1 (element Gauss, "Standard Gauss (Ref)", Sec. 3.1) and O2
(row-wise WQ/DWQ, Sec. 1-2 and Eq. 1) formation, and for the adjoint."""
import numpy as np
import pytest

from oracle.formation import OracleMesh
from oracle.geometry import F_INT, F_CUT
from oracle import adjoint
from tests.exact1d import exact_inner


def _greville(U, p):
    n = len(U) - p - 1
    return np.array([np.mean(U[i + 1:i + p + 1]) for i in range(n)])


@pytest.mark.parametrize("p", [2, 3])
def test_o1_full_cube_kronecker(p):
    """phi = -1, c = 1: M = M1 (x) M1 (x) M1 and K = K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1
    with 1D Gram matrices from exact piecewise-polynomial integrals."""
    n_el = (4, 3, 5)
    m = OracleMesh(dict(n_el=n_el, p=p, ls="full", octree_depth=1, coef="const", coef_const=1.0))
    M1 = [np.array([[exact_inner(s.U, p, i, j) for j in range(s.n)] for i in range(s.n)]) for s in m.spaces]
    K1 = [np.array([[exact_inner(s.U, p, i, j, 1) for j in range(s.n)] for i in range(s.n)]) for s in m.spaces]
    Mfull = np.kron(M1[2], np.kron(M1[1], M1[0]))
    Kfull = (np.kron(M1[2], np.kron(M1[1], K1[0])) + np.kron(M1[2], np.kron(K1[1], M1[0]))
             + np.kron(K1[2], np.kron(M1[1], M1[0])))
    g = m.geo
    for op, ref in (("mass", Mfull), ("stiffness", Kfull)):
        v = m.form_o1(op)
        for i in range(len(g.rowptr) - 1):
            cols = g.colind[g.rowptr[i]:g.rowptr[i + 1]]
            r = ref[i, cols]
            assert np.max(np.abs(v[g.rowptr[i]:g.rowptr[i + 1]] - r)) <= 1e-14 * np.max(np.abs(ref[i]))
            # the pattern holds every structural nonzero of the row
            assert abs(np.abs(ref[i]).sum() - np.abs(r).sum()) <= 1e-14 * np.abs(ref[i]).sum()


def test_o1_row_sums_and_constants():
    """c = 1: interior mass row sums equal int B_i = prod_d (U_{i+p+1} - U_i)/(p+1);
    stiffness rows annihilate constants for any c; total mass equals vol(Omega_h)."""
    desc = dict(n_el=(8, 8, 8), p=3, ls="ball", balls=[(0.52, 0.47, 0.5, 0.41)], octree_depth=2,
                coef="const", coef_const=1.0)
    m = OracleMesh(desc)
    g = m.geo
    M = m.form_o1("mass")
    p = m.p
    for i in np.nonzero(g.fclass == F_INT)[0]:
        idx = g.unravel_fn(i)
        ref = np.prod([(s.U[idx[d] + p + 1] - s.U[idx[d]]) / (p + 1) for d, s in enumerate(m.spaces)])
        assert abs(M[g.rowptr[i]:g.rowptr[i + 1]].sum() - ref) <= 1e-14 * ref
    assert abs(M.sum() - g.domain_volume()) <= 1e-13 * g.domain_volume()
    m2 = OracleMesh(dict(desc, coef="analytic"), geometry=g)
    for form in (m2.form_o1("stiffness"),
                 np.concatenate([v for _, v in sorted(m2.form_o2("stiffness").items())])):
        for i in np.nonzero(g.active)[0]:
            row = form[g.rowptr[i]:g.rowptr[i + 1]] if len(form) == g.rowptr[-1] else None
            if row is None:
                continue
            assert abs(row.sum()) <= 1e-13 * np.abs(row).sum()


@pytest.mark.parametrize("desc", [
    dict(n_el=(8, 8, 8), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, 0.4)], octree_depth=3),
    dict(n_el=(9, 7, 8), p=3, ls="plane", plane_pt=(0.1, 0.6, 0.3), plane_n=(0.5, -0.2, 0.9), octree_depth=2),
    dict(n_el=(6, 6, 7), p=4, ls="full", octree_depth=1),
    dict(n_el=(12, 12, 12), p=5, ls="ball", balls=[(0.45, 0.5, 0.55, 0.42)], octree_depth=1),
])
@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_o2_equals_o1_for_constant_coefficient(desc, op):
    """WQ/DWQ rules integrate products of the test function with trial functions exactly,
    so with a constant coefficient the method reproduces the Gauss matrix row by row."""
    m = OracleMesh(dict(desc, coef="const", coef_const=2.5))
    g = m.geo
    v1 = m.form_o1(op)
    rows = m.form_o2(op)
    n_int = n_box = 0
    for i, v in rows.items():
        r = v1[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.linalg.norm(v - r) <= 1e-13 * np.linalg.norm(r), i
        n_int += g.fclass[i] == F_INT
        n_box += g.fclass[i] == F_CUT and g.box(i) is not None
    if desc["ls"] != "full":
        assert n_box > 0
    else:
        assert n_int > 0


def test_o2_variable_coefficient_converges():
    """With variable c the method differs from Gauss by quadrature error only: the row
    sums approach int c B_i (reference: 12-point Gauss per element, numpy nodes) as h
    shrinks."""
    p = 3
    errs = []
    for ne in (6, 12, 24):
        m = OracleMesh(dict(n_el=(ne, ne, ne), p=p, ls="full", octree_depth=1, coef="analytic"))
        g = m.geo
        xg, wg = np.polynomial.legendre.leggauss(12)
        worst = 0.0
        for i in np.nonzero(g.fclass == F_INT)[0][::max(1, ne // 3)]:
            idx = g.unravel_fn(i)
            cols, vals = m.row_o2(int(i), "mass")
            pts, wts = [], []
            for d, s in enumerate(m.spaces):
                a, b = s.supp_elems(idx[d])
                t = np.concatenate([0.5 * (s.xb[e] + s.xb[e + 1]) + 0.5 * (s.xb[e + 1] - s.xb[e]) * xg
                                    for e in range(a, b + 1)])
                w = np.concatenate([0.5 * (s.xb[e + 1] - s.xb[e]) * wg for e in range(a, b + 1)])
                N = np.array([__import__("scipy").interpolate.BSpline(s.U, np.eye(s.n)[idx[d]], p)(t)])[0]
                pts.append(t)
                wts.append(w * N)
            T = np.meshgrid(*pts, indexing="ij")
            W = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
            ref = np.sum(W * m.coef(*T))
            worst = max(worst, abs(vals.sum() - ref) / abs(ref))
        errs.append(worst)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4
    # high-order convergence in h (a wrong point, weight or index gives an O(1) error)
    assert np.log2(errs[1] / errs[2]) > 3.0


@pytest.mark.parametrize("p", [2, 3])
def test_o1_brute_force_tiny_mesh(p):
    """2^3 mesh, ball domain, c linear in x (B-spline with Greville coefficients): c B_i B_j
    has degree <= 2p+1 per direction, so the (p+1)-point pieces agree with a 20-point Gauss
    rule per piece evaluated through scipy's B-splines."""
    from scipy.interpolate import BSpline
    desc = dict(n_el=(2, 2, 2), p=p, ls="ball", balls=[(0.45, 0.55, 0.5, 0.37)], octree_depth=3)
    base = OracleMesh(dict(desc, coef="const"))
    s0 = base.spaces[0]
    gr = _greville(s0.U, p)
    n = s0.n
    ck = np.broadcast_to(gr[None, None, :], (n, n, n)).ravel()
    m = OracleMesh(dict(desc, coef="bspline", coef_bspline=ck), geometry=base.geo)
    g = m.geo
    for op in ("mass", "stiffness"):
        v = m.form_o1(op)
        xg, wg = np.polynomial.legendre.leggauss(20)
        ref = {}
        boxes = []
        for e in range(len(g.state)):
            e1, e2, e3 = g.unravel_elem(e)
            if g.state[e] == 1:
                boxes.append(g.element_box(e1, e2, e3))
            elif g.state[e] == 2:
                boxes += [g.piece_box(pc) for pc in g.pieces[e]]
        B = [[BSpline(s.U, np.eye(s.n)[k], p) for k in range(s.n)] for s in m.spaces]
        acc = np.zeros((n ** 3, n ** 3))
        for bx in boxes:
            pts, wts = [], []
            for (a, b) in bx:
                pts.append(0.5 * (a + b) + 0.5 * (b - a) * xg)
                wts.append(0.5 * (b - a) * wg)
            T = np.meshgrid(*pts, indexing="ij")
            W = (wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]).ravel()
            c = T[0].ravel()
            vals = [np.array([B[d][k](pts[d]) for k in range(n)]) for d in range(3)]
            ders = [np.array([B[d][k].derivative()(pts[d]) for k in range(n)]) for d in range(3)]
            terms = [None] if op == "mass" else [0, 1, 2]
            for dd in terms:
                F = [ders[d] if dd == d else vals[d] for d in range(3)]
                Phi = np.einsum("ax,by,cz->cbaxyz", F[0], F[1], F[2]).reshape(n ** 3, -1)
                acc += (Phi * (W * c)[None, :]) @ Phi.T
        for i in np.nonzero(g.active)[0]:
            cols = g.colind[g.rowptr[i]:g.rowptr[i + 1]]
            r = acc[i, cols]
            assert np.max(np.abs(v[g.rowptr[i]:g.rowptr[i + 1]] - r)) <= 1e-13 * np.max(np.abs(r))


def test_adjoint_identities():
    """J = lambda^T A(c) u is linear in c: Euler identity sum_k c_k dJ/dc_k = J, and dJ/dc_k
    equals J evaluated with c replaced by the single basis function N_k."""
    rng = np.random.default_rng(5)
    p, ne = 2, 6
    n = ne + p
    ck = np.exp(0.5 * rng.standard_normal(n ** 3))
    desc = dict(n_el=(ne, ne, ne), p=p, ls="ball", balls=[(0.5, 0.5, 0.5, 0.37)], octree_depth=2,
                coef="bspline", coef_bspline=ck)
    m = OracleMesh(desc)
    lam, u = rng.standard_normal(n ** 3), rng.standard_normal(n ** 3)
    for op in ("mass", "stiffness"):
        grad = adjoint.gradient(m, op, lam, u)
        J = adjoint.bilinear(m, op, lam, u)
        assert abs(np.dot(ck, grad) - J) <= 1e-12 * abs(J)
        nz = np.nonzero(np.abs(grad) > 1e-3 * np.max(np.abs(grad)))[0]
        for k in rng.choice(nz, 4, replace=False):
            ek = np.zeros(n ** 3)
            ek[k] = 1.0
            mk = OracleMesh(dict(desc, coef_bspline=ek), geometry=m.geo)
            Jk = adjoint.bilinear(mk, op, lam, u)
            assert abs(grad[k] - Jk) <= 1e-12 * np.max(np.abs(grad))
