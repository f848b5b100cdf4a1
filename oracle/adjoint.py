"""Oracle adjoint: dJ/dc for J = lambda^T A(c) u with c = sum_k c_k N_k a B-spline field.
Test infrastructure only (see ``oracle/__init__``).

Every entry of A (method O2) is a finite quadrature sum that is linear in c:
A_ij = sum_x omega_i(x) c(x) Phi_j(x), with omega_i the test-function-folded weight of
row i at point x (a WQ / DWQ tensor weight, or w_g Phi_i(x_g) at a Gauss point).  Hence
J = sum_i lambda_i sum_x omega_i(x) c(x) sum_{j in row i} u_j Phi_j(x) and
dJ/dc_k = sum_i lambda_i sum_x omega_i(x) N_k(x) sum_{j in row i} u_j Phi_j(x).
This module evaluates that last line point by point.  Stiffness carries three terms,
one per direction d, with Phi = dB/dx_d on both sides.  (The coefficient-field gradient
is the paper-independent extension that the adjoint kernels implement.)
"""
import numpy as np

from .formation import OracleMesh, bspline_field, bspline_scatter
from .geometry import E_IN, E_CUT, F_INT, F_CUT


def gradient(mesh: OracleMesh, op, lam, u):
    """dJ/dc_k for all n1*n2*n3 coefficients (index k = k1 + n1 (k2 + n2 k3))."""
    geo = mesh.geo
    p = mesh.p
    n1, n2, n3 = mesh.n
    lam = np.asarray(lam, float).ravel()
    ucoef = np.asarray(u, float).reshape(n3, n2, n1)
    grad = np.zeros((n3, n2, n1))
    terms = [(None, ("00", "00", "00"))] if op == "mass" else \
        [(0, ("11", "00", "00")), (1, ("00", "11", "00")), (2, ("00", "00", "11"))]
    # (1) weighted-quadrature points of interior rows and of DWQ boxes
    for i in np.nonzero(geo.active)[0]:
        i = int(i)
        cls = geo.fclass[i]
        box = geo.box(i) if cls == F_CUT else None
        if not (cls == F_INT or box is not None):
            continue
        idx = geo.unravel_fn(i)
        for dd, kinds in terms:
            rules = mesh._wq_term_rules(idx, box, kinds)
            pts = [mesh.spaces[d].t_sup[rules[d][0]] for d in range(3)]
            T1, T2, T3 = np.meshgrid(pts[0], pts[1], pts[2], indexing="ij")
            W = rules[0][1][:, None, None] * rules[1][1][None, :, None] * rules[2][1][None, None, :]
            Uq = bspline_field(mesh.spaces, ucoef, T1, T2, T3, deriv_dir=dd)
            bspline_scatter(mesh.spaces, (T1.ravel(), T2.ravel(), T3.ravel()),
                            lam[i] * (W * Uq).ravel(), grad)
    # (2) Gauss points, element by element: the rows that integrate element e with Gauss
    # points are all active rows whose support holds e when e is cut, and the cut rows
    # whose DWQ box does not hold e when e is inside.
    for e in range(len(geo.state)):
        st = geo.state[e]
        if st not in (E_IN, E_CUT):
            continue
        e1, e2, e3 = geo.unravel_elem(e)
        if st == E_IN:
            X, W = mesh.element_points(e1, e2, e3)
        else:
            X, W = mesh.cut_points(e)
        lam_e = np.zeros((n3, n2, n1))
        any_row = False
        for a3 in range(p + 1):
            for a2 in range(p + 1):
                for a1 in range(p + 1):
                    i1, i2, i3 = e1 + a1, e2 + a2, e3 + a3
                    i = geo.fn_index(i1, i2, i3)
                    if geo.fclass[i] != F_CUT:
                        continue
                    if st == E_IN:
                        box = geo.box(i)
                        if box is not None:
                            d, b, side = box
                            ed = (e1, e2, e3)[d]
                            if (side == 0 and ed < b) or (side == 1 and ed >= b):
                                continue
                    lam_e[i3, i2, i1] = lam[i]
                    any_row = True
        if not any_row:
            continue
        for dd, _ in terms:
            Lx = bspline_field(mesh.spaces, lam_e, X[0], X[1], X[2], deriv_dir=dd)
            Ux = bspline_field(mesh.spaces, ucoef, X[0], X[1], X[2], deriv_dir=dd)
            bspline_scatter(mesh.spaces, X, W * Lx * Ux, grad)
    return grad.ravel()


def bilinear(mesh: OracleMesh, op, lam, u, values=None):
    """J = lambda^T A u with A formed by O2 (or the given CSR values on the pattern)."""
    geo = mesh.geo
    lam = np.asarray(lam, float).ravel()
    u = np.asarray(u, float).ravel()
    if values is None:
        rows = mesh.form_o2(op)
        J = 0.0
        for i, v in rows.items():
            cols = geo.colind[geo.rowptr[i]:geo.rowptr[i + 1]]
            J += lam[i] * np.dot(v, u[cols])
        return J
    J = 0.0
    for i in np.nonzero(geo.active)[0]:
        s, t = geo.rowptr[i], geo.rowptr[i + 1]
        J += lam[i] * np.dot(values[s:t], u[geo.colind[s:t]])
    return J
