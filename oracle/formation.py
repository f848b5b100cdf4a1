"""Oracle formation of mass and Laplace-stiffness matrices on the CSR pattern.
Test infrastructure only (see ``oracle/__init__``).

O1  "Standard Gauss (Ref)" (Sec. 3.1): element loop with (p+1)^3 Gauss points per
    inside element and per octree piece of a cut element.  This is the reference
    integral over the discrete domain Omega_h.
O2  the paper's method (Sec. 1 ingredients, Sec. 2.2, Eq. 1), row by row:
    * interior row i: weighted quadrature on the tensor grid of WQ points,
      A_ij = sum_q w_i1(q1) w_i2(q2) w_i3(q3) c(x_q) B_j(x_q) (mass); stiffness is the
      sum over d of the same with the derivative rule w11 and B_j' in direction d;
    * cut row i (Eq. 1 split of the support): the regular part S^r is the DWQ box
      (one-sided DWQ rule in direction d, standard WQ in the other two) when a box
      exists, every other inside support element is integrated with element Gauss
      points, and every cut support element with the Gauss points of its octree
      pieces.  Without a box the row is integrated entirely with Gauss points.
Both are written as plain quadrature-point sums (a point-by-column matrix product
per row or element); no sum factorisation.
"""
import numpy as np

from .bspline import basis_all, basis_local, gauss_legendre
from .wq import Space1D
from .geometry import Geometry, E_IN, E_CUT, F_INT, F_CUT, _g


def _local_basis_at(space, v, deriv):
    """For points v (1D): element index e of each point and the p+1 values (or first
    derivatives) of functions e..e+p, shape (p+1, len(v))."""
    p = space.p
    e = np.clip(np.searchsorted(space.xb, v, side="right") - 1, 0, space.n_el - 1)
    out = np.zeros((p + 1, len(v)))
    for ee in np.unique(e):
        sel = e == ee
        N, dN = basis_local(space.U, p, ee + p, v[sel])
        out[:, sel] = dN if deriv else N
    return e, out


def bspline_field(spaces, ck, x, y, z, deriv_dir=None):
    """sum_k ck[k3, k2, k1] N_k1(x) N_k2(y) N_k3(z) pointwise (or its partial derivative
    in direction deriv_dir), summing the (p+1)^3 nonzero terms of each point."""
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    shp = x.shape
    p = spaces[0].p
    P = x.size
    Nl, El = [], []
    for d, (s, v) in enumerate(zip(spaces, (x, y, z))):
        e, Nv = _local_basis_at(s, v.ravel(), deriv_dir == d)
        Nl.append(Nv)
        El.append(e)
    out = np.zeros(P)
    for a3 in range(p + 1):
        for a2 in range(p + 1):
            for a1 in range(p + 1):
                c = ck[El[2] + a3, El[1] + a2, El[0] + a1]
                out += c * Nl[0][a1] * Nl[1][a2] * Nl[2][a3]
    return out.reshape(shp)


def bspline_scatter(spaces, X, f, out):
    """out[k3, k2, k1] += sum_x f(x) N_k1(x1) N_k2(x2) N_k3(x3) (transpose of bspline_field)."""
    p = spaces[0].p
    Nl, El = [], []
    for d in range(3):
        e, Nv = _local_basis_at(spaces[d], np.asarray(X[d], float).ravel(), False)
        Nl.append(Nv)
        El.append(e)
    f = np.asarray(f, float).ravel()
    for a3 in range(p + 1):
        for a2 in range(p + 1):
            for a1 in range(p + 1):
                np.add.at(out, (El[2] + a3, El[1] + a2, El[0] + a1), f * Nl[0][a1] * Nl[1][a2] * Nl[2][a3])


class Coefficient:
    """Coefficient field c(x): constant, the analytic field 1 + 0.5 sin(2 pi x) cos(2 pi y) z,
    or a B-spline sum_k c_k N_k(x) on the mesh's own knots and degree
    (coefficients indexed k = k1 + n1 (k2 + n2 k3))."""

    def __init__(self, desc, spaces):
        self.kind = _g(desc, "coef", "const")
        self.c0 = float(_g(desc, "coef_const", 1.0))
        self.spaces = spaces
        if self.kind == "bspline":
            n1, n2, n3 = (s.n for s in spaces)
            self.ck = np.asarray(_g(desc, "coef_bspline"), dtype=np.float64).reshape(n3, n2, n1)

    def __call__(self, x, y, z):
        x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
        if self.kind == "const":
            return np.full(x.shape, self.c0)
        if self.kind == "analytic":
            return 1.0 + 0.5 * np.sin(2.0 * np.pi * x) * np.cos(2.0 * np.pi * y) * z
        if self.kind == "bspline":
            return bspline_field(self.spaces, self.ck, x, y, z)
        raise ValueError(self.kind)


class OracleMesh:
    """Spaces, rules, geometry and coefficient for one mesh description."""

    def __init__(self, desc, geometry=None):
        self.desc = desc
        self.p = int(_g(desc, "p"))
        n_el = tuple(int(v) for v in _g(desc, "n_el"))
        lo = tuple(float(v) for v in _g(desc, "lo", (0.0, 0.0, 0.0)))
        hi = tuple(float(v) for v in _g(desc, "hi", (1.0, 1.0, 1.0)))
        self.spaces = [Space1D(n_el[d], self.p, lo[d], hi[d]) for d in range(3)]
        self.geo = geometry if geometry is not None else Geometry(desc)
        self.coef = Coefficient(desc, self.spaces)
        self.n = tuple(s.n for s in self.spaces)
        self.xg, self.wg = gauss_legendre(self.p + 1)

    # ---- basis helpers ---------------------------------------------------------------
    def basis_1d(self, d, t):
        """All functions of direction d at points t: (N, dN) of shape (n_d, len(t))."""
        s = self.spaces[d]
        return basis_all(s.U, s.p, t)

    def band(self, d, i):
        """Column range of the band of row index i in direction d (clipped)."""
        return max(0, i - self.p), min(self.n[d] - 1, i + self.p)

    # ---- point sets with test-function-folded weights ----------------------------------
    def _wq_term_rules(self, idx, box, kind_by_dir):
        """Per-direction (superset idx, weights) for one stiffness/mass term.
        kind_by_dir[d] in {'00','11'}.  With a box (d, b, side) the DWQ rule is used in d."""
        out = []
        for d in range(3):
            s = self.spaces[d]
            if box is not None and box[0] == d:
                w = s.dwq_rule(idx[d], box[1], box[2], kind_by_dir[d])
                Q = np.nonzero(w)[0]
                # keep structurally kept-side points even when a weight is exactly zero
                e_lo, e_hi = s.supp_elems(idx[d])
                b, side = box[1], box[2]
                kept = list(range(e_lo, b)) if side == 0 else list(range(b, e_hi + 1))
                layout = s.wq_mask | (s.elem_of_sup == b - 1) | (s.elem_of_sup == b)
                Q = np.nonzero(np.isin(s.elem_of_sup, kept) & layout)[0]
                out.append((Q, w[Q]))
            else:
                out.append(s.std_rule(idx[d], kind_by_dir[d]))
        return out

    def _grid_sum(self, rules, deriv_dir, i, cols_rng):
        """sum over the tensor grid of rules of W(q) c(x_q) Phi_j(x_q) for all band columns j.
        deriv_dir: None (mass: Phi_j = B_j) or d (Phi_j = B_j with the derivative in d)."""
        pts = [self.spaces[d].t_sup[rules[d][0]] for d in range(3)]
        T1, T2, T3 = np.meshgrid(pts[0], pts[1], pts[2], indexing="ij")
        W = (rules[0][1][:, None, None] * rules[1][1][None, :, None] * rules[2][1][None, None, :])
        F = (W * self.coef(T1, T2, T3)).ravel()  # point order (q1, q2, q3), q3 fastest
        Bd = []
        for d in range(3):
            N, dN = self.basis_1d(d, pts[d])
            a, b = cols_rng[d]
            Bd.append((dN if deriv_dir == d else N)[a:b + 1])  # (nj_d, nq_d)
        # Phi[q, j] with q = (q1, q2, q3) and j = (j3, j2, j1) (j1 fastest)
        Phi = np.einsum("ax,by,cz->xyzcba", Bd[0], Bd[1], Bd[2]).reshape(F.size, -1)
        return F @ Phi

    def _points_sum(self, X, W, i_idx, cols_rng, op):
        """Gauss-point sum over scattered points X (3, m) with weights W (m):
        sum_g W_g c(x_g) Phi_i(x_g) Phi_j(x_g) for all band columns j (order j3, j2, j1)."""
        c = self.coef(X[0], X[1], X[2])
        Nd, dNd = [], []
        for d in range(3):
            N, dN = self.basis_1d(d, X[d])
            Nd.append(N)
            dNd.append(dN)
        out = 0.0
        terms = [None] if op == "mass" else [0, 1, 2]
        for dd in terms:
            fi = np.ones(X.shape[1])
            Bj = []
            for d in range(3):
                M = dNd[d] if dd == d else Nd[d]
                fi = fi * M[i_idx[d]]
                a, b = cols_rng[d]
                Bj.append(M[a:b + 1])
            Phi = np.einsum("ag,bg,cg->gcba", Bj[0], Bj[1], Bj[2]).reshape(X.shape[1], -1)
            out = out + (W * c * fi) @ Phi
        return out

    def element_points(self, e1, e2, e3):
        """(p+1)^3 Gauss points and weights of a whole element (the superset points)."""
        ts, ws = [], []
        for d, e in enumerate((e1, e2, e3)):
            s = self.spaces[d]
            sl = slice(e * (self.p + 1), (e + 1) * (self.p + 1))
            ts.append(s.t_sup[sl])
            ws.append(s.w_sup[sl])
        return self._tensor_points(ts, ws)

    def piece_points(self, piece):
        """(p+1)^3 Gauss points and weights of an octree piece."""
        ts, ws = [], []
        for (a, b) in self.geo.piece_box(piece):
            mid, half = 0.5 * (a + b), 0.5 * (b - a)
            ts.append(mid + half * self.xg)
            ws.append(half * self.wg)
        return self._tensor_points(ts, ws)

    @staticmethod
    def _tensor_points(ts, ws):
        T1, T2, T3 = np.meshgrid(ts[0], ts[1], ts[2], indexing="ij")
        W = ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
        return np.stack([T1.ravel(), T2.ravel(), T3.ravel()]), W.ravel()

    def cut_points(self, e):
        """All Gauss points (3, m) and weights (m) of the pieces of cut element e."""
        if not hasattr(self, "_cut_pts"):
            self._cut_pts = {}
        if e not in self._cut_pts:
            pcs = self.geo.pieces.get(e, [])
            if not pcs:
                self._cut_pts[e] = None
                return None
            boxes = np.array([self.geo.piece_box(pc) for pc in pcs])  # (np, 3, 2)
            mid = 0.5 * (boxes[:, :, 0] + boxes[:, :, 1])
            half = 0.5 * (boxes[:, :, 1] - boxes[:, :, 0])
            t = mid[:, :, None] + half[:, :, None] * self.xg[None, None, :]  # (np, 3, p+1)
            w = half[:, :, None] * self.wg[None, None, :]
            q = self.p + 1
            X = np.stack([np.broadcast_to(t[:, 0, :, None, None], (len(pcs), q, q, q)),
                          np.broadcast_to(t[:, 1, None, :, None], (len(pcs), q, q, q)),
                          np.broadcast_to(t[:, 2, None, None, :], (len(pcs), q, q, q))]).reshape(3, -1)
            W = (w[:, 0, :, None, None] * w[:, 1, None, :, None] * w[:, 2, None, None, :]).ravel()
            self._cut_pts[e] = (X, W)
        return self._cut_pts[e]

    # ---- O2: one row ------------------------------------------------------------------
    def row_band_o2(self, i, op, variant="dwq"):
        """Dense band of row i (order j3, j2, j1 over the clipped band), method O2.
        variant "hybrid" (Sec. 3.1, "Hybrid Gauss"): cut rows take no DWQ box, so their whole
        regular part is integrated with element Gauss points."""
        geo = self.geo
        idx = geo.unravel_fn(i)
        cols_rng = [self.band(d, idx[d]) for d in range(3)]
        cls = geo.fclass[i]
        terms = [(None, ("00", "00", "00"))] if op == "mass" else \
            [(0, ("11", "00", "00")), (1, ("00", "11", "00")), (2, ("00", "00", "11"))]
        box = None
        if cls == F_CUT and variant == "dwq":
            box = geo.box(i)
        V = 0.0
        if cls == F_INT or box is not None:
            for deriv_dir, kinds in terms:
                rules = self._wq_term_rules(idx, box, kinds)
                V = V + self._grid_sum(rules, deriv_dir, i, cols_rng)
        if cls == F_CUT:
            V = V + self.gauss_part(i, idx, box, cols_rng, op)
        return V, cols_rng

    def gauss_part(self, i, idx, box, cols_rng, op):
        """Gauss points over the inside support elements outside the box and the pieces
        of every cut support element: sum over those elements of the element Gauss sums
        int_e c Phi_i Phi_j (row a(i) of the element's Gauss matrix)."""
        geo = self.geo
        p = self.p
        rng = [geo.supp(d, idx[d]) for d in range(3)]
        w = [cols_rng[d][1] - cols_rng[d][0] + 1 for d in range(3)]
        V = np.zeros(w[0] * w[1] * w[2])
        for e3 in range(rng[2][0], rng[2][1] + 1):
            for e2 in range(rng[1][0], rng[1][1] + 1):
                for e1 in range(rng[0][0], rng[0][1] + 1):
                    e = geo.elem_index(e1, e2, e3)
                    st = geo.state[e]
                    if st == E_IN:
                        if box is not None:
                            d, b, side = box
                            ed = (e1, e2, e3)[d]
                            if (side == 0 and ed < b) or (side == 1 and ed >= b):
                                continue  # inside the DWQ box
                    elif st != E_CUT:
                        continue
                    Me = self.element_matrix(e, op)
                    a = (idx[0] - e1) + (p + 1) * ((idx[1] - e2) + (p + 1) * (idx[2] - e3))
                    row = Me[a].reshape(p + 1, p + 1, p + 1)  # (b3, b2, b1)
                    o = [(e1, e2, e3)[d] - cols_rng[d][0] for d in range(3)]
                    Vv = V.reshape(w[2], w[1], w[0])
                    Vv[o[2]:o[2] + p + 1, o[1]:o[1] + p + 1, o[0]:o[0] + p + 1] += row
        return V

    def element_matrix(self, e, op):
        """Gauss matrix of element e (inside: (p+1)^3 element Gauss points; cut: the Gauss
        points of its octree pieces): M[a, b] = sum_g w_g c(x_g) Phi_a(x_g) Phi_b(x_g) over the
        (p+1)^3 local functions, local order (a3, a2, a1)."""
        if not hasattr(self, "_emats"):
            self._emats = {}
        key = (e, op)
        if key in self._emats:
            return self._emats[key]
        geo = self.geo
        p = self.p
        e1, e2, e3 = geo.unravel_elem(e)
        if geo.state[e] == E_IN:
            X, W = self.element_points(e1, e2, e3)
        else:
            X, W = self.cut_points(e)
        c = self.coef(X[0], X[1], X[2])
        Nd, dNd = [], []
        for d, ed in enumerate((e1, e2, e3)):
            N, dN = basis_local(self.spaces[d].U, p, ed + p, X[d])
            Nd.append(N)
            dNd.append(dN)
        terms = [None] if op == "mass" else [0, 1, 2]
        Me = 0.0
        for dd in terms:
            M = [dNd[d] if dd == d else Nd[d] for d in range(3)]
            Phi = np.einsum("ag,bg,cg->cbag", M[0], M[1], M[2]).reshape(-1, X.shape[1])
            Me = Me + (Phi * (W * c)[None, :]) @ Phi.T
        self._emats[key] = Me
        return Me

    def row_o2(self, i, op, variant="dwq"):
        """(columns, values) of row i on the CSR pattern, method O2."""
        V, cols_rng = self.row_band_o2(i, op, variant)
        return self._band_to_row(i, V, cols_rng)

    def _band_to_row(self, i, V, cols_rng):
        geo = self.geo
        n1, n2, _ = self.n
        (a1, b1), (a2, b2), (a3, b3) = cols_rng
        J1, J2, J3 = np.meshgrid(np.arange(a1, b1 + 1), np.arange(a2, b2 + 1), np.arange(a3, b3 + 1),
                                 indexing="ij")
        jband = (J1 + n1 * (J2 + n2 * J3)).transpose(2, 1, 0).ravel()  # (j3, j2, j1) order
        cols = geo.colind[geo.rowptr[i]:geo.rowptr[i + 1]]
        pos = {int(j): k for k, j in enumerate(jband)}
        V = np.broadcast_to(np.asarray(V, dtype=np.float64), (len(jband),))
        vals = np.array([V[pos[int(j)]] for j in cols])
        return cols, vals

    def form_o2(self, op, rows=None, variant="dwq"):
        """Values on the CSR pattern for the given rows (all active rows by default).
        Returns a dict row -> values (pattern order)."""
        geo = self.geo
        if rows is None:
            rows = np.nonzero(geo.active)[0]
        return {int(i): self.row_o2(int(i), op, variant)[1] for i in rows}

    # ---- load vector by the same rules ---------------------------------------------------
    def source(self, src):
        """Load-vector source f: "coef" (the coefficient field c) or "paper"
        (f = sin(2xz) cos(3yz), the target function of the paper's experiment, Sec. 3.1)."""
        if src == "coef":
            return self.coef
        if src == "paper":
            return lambda x, y, z: np.sin(2.0 * x * z) * np.cos(3.0 * y * z)
        raise ValueError(src)

    def row_load_o2(self, i, src="coef", variant="dwq"):
        """b_i, the rules of row i applied to f: interior rows sum_q w_i1 w_i2 w_i3 f(x_q)
        over the tensor grid of their WQ rules (the test function is folded into the weights,
        Sec. 1); cut rows the DWQ box part plus f B_i at the Gauss points of the inside
        support elements outside the box and of the octree pieces of the cut ones (Eq. 1)."""
        geo = self.geo
        f = self.source(src)
        cls = geo.fclass[i]
        if cls not in (F_INT, F_CUT):
            return 0.0
        idx = geo.unravel_fn(i)
        box = geo.box(i) if (cls == F_CUT and variant == "dwq") else None
        b = 0.0
        if cls == F_INT or box is not None:
            rules = self._wq_term_rules(idx, box, ("00", "00", "00"))
            pts = [self.spaces[d].t_sup[rules[d][0]] for d in range(3)]
            T1, T2, T3 = np.meshgrid(pts[0], pts[1], pts[2], indexing="ij")
            W = (rules[0][1][:, None, None] * rules[1][1][None, :, None] * rules[2][1][None, None, :])
            b += float(np.sum(W * f(T1, T2, T3)))
        if cls == F_CUT:
            rng = [geo.supp(d, idx[d]) for d in range(3)]
            for e3 in range(rng[2][0], rng[2][1] + 1):
                for e2 in range(rng[1][0], rng[1][1] + 1):
                    for e1 in range(rng[0][0], rng[0][1] + 1):
                        e = geo.elem_index(e1, e2, e3)
                        st = geo.state[e]
                        if st == E_IN:
                            if box is not None:
                                d, bb, side = box
                                ed = (e1, e2, e3)[d]
                                if (side == 0 and ed < bb) or (side == 1 and ed >= bb):
                                    continue
                            X, W = self.element_points(e1, e2, e3)
                        elif st == E_CUT:
                            X, W = self.cut_points(e)
                        else:
                            continue
                        Bi = np.ones(X.shape[1])
                        for d in range(3):
                            N, _ = basis_local(self.spaces[d].U, self.p, (e1, e2, e3)[d] + self.p, X[d])
                            Bi = Bi * N[idx[d] - (e1, e2, e3)[d]]
                        b += float(np.sum(W * f(X[0], X[1], X[2]) * Bi))
        return b

    def load_o2(self, rows=None, src="coef", variant="dwq"):
        """Load values of the given rows (all active rows by default), as an array."""
        geo = self.geo
        if rows is None:
            rows = np.nonzero(geo.active)[0]
        return np.array([self.row_load_o2(int(i), src, variant) for i in rows])

    # ---- O1: element loop --------------------------------------------------------------
    def form_o1(self, op):
        """Element-wise Gauss formation; returns CSR values on the pattern (all rows)."""
        geo = self.geo
        p = self.p
        n1, n2, _ = self.n
        nnz = int(geo.rowptr[-1])
        vals = np.zeros(nnz)
        pos = {}
        for e in range(len(geo.state)):
            if geo.state[e] not in (E_IN, E_CUT):
                continue
            e1, e2, e3 = geo.unravel_elem(e)
            Me = self.element_matrix(e, op)
            loc = [(e1 + a1) + n1 * ((e2 + a2) + n2 * (e3 + a3))
                   for a3 in range(p + 1) for a2 in range(p + 1) for a1 in range(p + 1)]
            for r, i in enumerate(loc):
                if i not in pos:
                    cols = geo.colind[geo.rowptr[i]:geo.rowptr[i + 1]]
                    pos[i] = {int(j): int(geo.rowptr[i]) + k for k, j in enumerate(cols)}
                pi = pos[i]
                for cidx, j in enumerate(loc):
                    vals[pi[j]] += Me[r, cidx]
        return vals
