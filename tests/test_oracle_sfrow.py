"""Pins for the C row oracle (oracle/sfrow.c): the row loop with sum factorisation (Sec. 1,
Table 2), the Hybrid Gauss and Standard Gauss variants (Sec. 3.1) and the load vector.

The C oracle is pinned to things other than itself:
  * the numpy O2 (plain quadrature-point loops, itself pinned in test_oracle_formation.py):
    the same sums in another order agree to rounding on every active row;
  * O1 (element Gauss): the Standard Gauss variant must reproduce its rows, and Hybrid Gauss
    rows of cut functions are pure Gauss sums, so they must equal O1's rows for any c;
  * closed forms and brute force for the load vector: with f = 1 an interior value is
    int B_i = prod_d (U_{i+p+1} - U_i) / (p+1); with f a B-spline of the mesh's own space the
    rules are exact (f B_i is a polynomial per element and f is a trial function), so every
    value equals a 20-point Gauss integral of f B_i over the discrete domain;
  * its Cox-de Boor values against scipy's B-splines.
"""
import numpy as np
import pytest

from oracle.formation import OracleMesh
from oracle.geometry import F_CUT, F_INT
from oracle.sfrow import RowOracle, basis_values

MESHES = {
    "ball_p2": dict(n_el=(8, 8, 8), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, 0.4)], octree_depth=3, coef="analytic"),
    "plane_p3": dict(n_el=(9, 7, 8), p=3, ls="plane", plane_pt=(0.1, 0.6, 0.3), plane_n=(0.5, -0.2, 0.9),
                     octree_depth=2, coef="analytic"),
    "full_p4": dict(n_el=(7, 6, 8), p=4, ls="full", octree_depth=1, coef="analytic"),
    "balls_p4": dict(n_el=(10, 9, 8), p=4, ls="balls", balls=[(0.3, 0.4, 0.5, 0.25), (0.65, 0.6, 0.45, 0.28)],
                     octree_depth=2, coef="analytic"),
    "gyroid_p2": dict(n_el=(10, 10, 10), p=2, ls="gyroid", gyroid_freq=6.0, gyroid_iso=0.3, octree_depth=2,
                      coef="const", coef_const=1.7),
}


def _bspline_coef(n_el, p, seed):
    n = [ne + p for ne in n_el]
    return np.exp(0.5 * np.random.default_rng(seed).standard_normal(n[0] * n[1] * n[2]))


def _worst(a, b):
    return max(np.linalg.norm(a[i] - v) / max(np.linalg.norm(v), 1e-300) for i, v in b.items())


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_c_rows_equal_numpy_o2(name, op):
    om = OracleMesh(MESHES[name])
    ref = om.form_o2(op)
    got = RowOracle(om).rows(op)
    assert set(got) == set(ref)
    assert _worst(got, ref) <= 1e-13


@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_c_rows_equal_numpy_o2_bspline_coefficient_p5(op):
    desc = dict(n_el=(10, 9, 11), p=5, ls="plane", plane_pt=(0.5, 0.45, 0.55), plane_n=(0.3, -0.2, 0.9),
                octree_depth=1, coef="bspline", coef_bspline=_bspline_coef((10, 9, 11), 5, 3))
    om = OracleMesh(desc)
    g = om.geo
    cuts = np.nonzero(g.fclass == F_CUT)[0]
    boxed = [int(i) for i in cuts if g.box(int(i)) is not None]
    assert boxed
    rows = list(np.nonzero(g.fclass == F_INT)[0][::7]) + list(cuts[::17]) + boxed[::max(1, len(boxed) // 12)]
    ref = om.form_o2(op, rows)
    assert _worst(RowOracle(om).rows(op, rows), ref) <= 1e-13


@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_hybrid_variant(op):
    """Hybrid Gauss: C equals numpy on every row; its cut rows are pure Gauss sums and equal
    O1's rows (variable c), while its interior rows stay the WQ rows of the method."""
    om = OracleMesh(MESHES["plane_p3"])
    g = om.geo
    ref = om.form_o2(op, variant="hybrid")
    got = RowOracle(om, variant="hybrid").rows(op)
    assert _worst(got, ref) <= 1e-13
    o1 = om.form_o1(op)
    dwq = om.form_o2(op)
    n_box = 0
    for i, v in ref.items():
        r1 = o1[g.rowptr[i]:g.rowptr[i + 1]]
        if g.fclass[i] == F_CUT:
            assert np.linalg.norm(v - r1) <= 1e-13 * np.linalg.norm(r1), i
            n_box += g.box(i) is not None
        else:
            assert np.array_equal(v, dwq[i])
    assert n_box > 0  # the variant differs from the method on these rows


@pytest.mark.parametrize("name", ["ball_p2", "plane_p3"])
@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_gauss_variant_equals_o1(name, op):
    om = OracleMesh(MESHES[name])
    g = om.geo
    o1 = om.form_o1(op)
    got = RowOracle(om, variant="gauss").rows(op)
    for i, v in got.items():
        r1 = o1[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.linalg.norm(v - r1) <= 1e-13 * np.linalg.norm(r1), i


def test_basis_values_match_scipy():
    from scipy.interpolate import BSpline
    from oracle.bspline import open_knots
    rng = np.random.default_rng(0)
    for p in (2, 3, 6):
        n_el = 7
        U = open_knots(n_el, p)
        n = n_el + p
        for x in rng.uniform(0, 1, 20):
            first, N, dN = basis_values(U, p, n_el, x)
            for r in range(p + 1):
                spl = BSpline(U, np.eye(n)[first + r], p)
                assert abs(N[r] - spl(x)) <= 1e-15
                assert abs(dN[r] - spl.derivative()(x)) <= 1e-12


def _brute_force_load(om, f, rows):
    """int over Omega_h of f B_i with 20-point Gauss per inside element and per octree piece,
    B_i by scipy."""
    from scipy.interpolate import BSpline
    g = om.geo
    xg, wg = np.polynomial.legendre.leggauss(20)
    boxes = []
    for e in range(len(g.state)):
        e1, e2, e3 = g.unravel_elem(e)
        if g.state[e] == 1:
            boxes.append(g.element_box(e1, e2, e3))
        elif g.state[e] == 2:
            boxes += [g.piece_box(pc) for pc in g.pieces[e]]
    out = np.zeros(len(rows))
    B = [[BSpline(s.U, np.eye(s.n)[k], s.p) for k in range(s.n)] for s in om.spaces]
    for bx in boxes:
        pts = [0.5 * (a + b) + 0.5 * (b - a) * xg for (a, b) in bx]
        wts = [0.5 * (b - a) * wg for (a, b) in bx]
        T = np.meshgrid(*pts, indexing="ij")
        W = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
        F = W * f(*T)
        for k, i in enumerate(rows):
            idx = g.unravel_fn(int(i))
            b = [B[d][idx[d]](pts[d]) for d in range(3)]
            out[k] += np.einsum("xyz,x,y,z->", F, b[0], b[1], b[2])
    return out


def test_load_vector_pins():
    """f = 1: interior values equal prod_d (U_{i+p+1} - U_i)/(p+1); every value equals the
    brute-force integral over the discrete domain.  f a B-spline of the space: WQ and DWQ
    are exact (exactness with the trial functions), so the values equal the brute-force
    integral of f B_i again.  C and numpy agree on every row for the paper's f too."""
    base = dict(n_el=(5, 4, 6), p=2, ls="plane", plane_pt=(0.5, 0.45, 0.55), plane_n=(0.3, -0.2, 0.9),
                octree_depth=2)
    om1 = OracleMesh(dict(base, coef="const", coef_const=1.0))
    g = om1.geo
    rows = np.nonzero(g.fclass != 0)[0]
    b_np = om1.load_o2(rows)
    b_c = RowOracle(om1).load(rows)
    assert np.max(np.abs(b_np - b_c)) <= 1e-14 * np.max(np.abs(b_np))
    p = om1.p
    n_box = 0
    for k, i in enumerate(rows):
        if g.fclass[i] == F_INT:
            idx = g.unravel_fn(int(i))
            ref = np.prod([(s.U[idx[d] + p + 1] - s.U[idx[d]]) / (p + 1) for d, s in enumerate(om1.spaces)])
            assert abs(b_np[k] - ref) <= 1e-14 * ref
        else:
            n_box += g.box(int(i)) is not None
    assert n_box > 0
    one = _brute_force_load(om1, lambda x, y, z: np.ones_like(x), rows)
    assert np.max(np.abs(b_np - one) / np.abs(one)) <= 1e-12
    ck = _bspline_coef(base["n_el"], p, 11)
    om2 = OracleMesh(dict(base, coef="bspline", coef_bspline=ck), geometry=g)
    b2 = RowOracle(om2).load(rows)
    ref2 = _brute_force_load(om2, om2.coef, rows)
    assert np.max(np.abs(b2 - ref2) / np.abs(ref2)) <= 1e-12
    bp = om2.load_o2(rows, src="paper")
    bpc = RowOracle(om2, src="paper").load(rows)
    assert np.max(np.abs(bp - bpc)) <= 1e-14 * np.max(np.abs(bp))
    # the variants: Gauss sums over the support of each row
    bg = RowOracle(om1, variant="gauss").load(rows)
    assert np.max(np.abs(bg - one) / np.abs(one)) <= 1e-12
    bh = RowOracle(om2, variant="hybrid", src="paper").load(rows)
    bhn = om2.load_o2(rows, src="paper", variant="hybrid")
    assert np.max(np.abs(bh - bhn)) <= 1e-14 * np.max(np.abs(bhn))
