"""Oracle weighted-quadrature (WQ) and discontinuous WQ (DWQ) rules.
Test infrastructure only (see ``oracle/__init__``).

Sec. 1 (WQ ingredient): a rule per test function B_i, with the test function
folded into the weights, such that sum_q w_i(q) B_j(t_q) = int B_i B_j for every
trial function B_j of the space.  Sec. 2.2 (last paragraph): the WQ points are a
subset of the element-wise Gauss points ("Gauss superset"), and when a rule's
elements all carry the full Gauss set the Gauss weights are used directly.
Sec. 2.2 steps 3-6: DWQ rules by knot insertion (subdivision matrix S), nested
points next to the artificial discontinuity, refined WQ weights, S^T combination;
weights on the far side of the discontinuity are zero.

Readings (the paper defers these details to its references):
* point subset: all p+1 Gauss points in the first and last element, Gauss
  indices {0, p} in every other element;
* weights: the minimum-Euclidean-norm solution of the exactness system
  (numpy lstsq, SVD based, rcond 1e-12); the w11 system (derivatives) is
  rank deficient by one because the derivatives of a partition of unity sum
  to zero, and the min-norm solution is still unique;
* nested points: all p+1 Gauss points of the two elements next to the
  discontinuity; the far side is dropped.
"""
import numpy as np

from .bspline import gauss_legendre, open_knots, element_bounds, basis_all, subdivision_matrix


class Space1D:
    """Univariate open-knot B-spline space of degree p with n_el uniform elements on [lo, hi],
    its Gauss superset (p+1 points per element) and the WQ point subset."""

    def __init__(self, n_el, p, lo=0.0, hi=1.0):
        self.n_el, self.p, self.lo, self.hi = int(n_el), int(p), float(lo), float(hi)
        self.n = self.n_el + self.p
        self.U = open_knots(self.n_el, self.p, self.lo, self.hi)
        self.xb = element_bounds(self.n_el, self.lo, self.hi)
        xg, wg = gauss_legendre(self.p + 1)
        self.xg, self.wg = xg, wg
        mid = 0.5 * (self.xb[:-1] + self.xb[1:])
        half = 0.5 * (self.xb[1:] - self.xb[:-1])
        self.t_sup = (mid[:, None] + half[:, None] * xg[None, :]).ravel()
        self.w_sup = (half[:, None] * wg[None, :]).ravel()
        self.elem_of_sup = np.repeat(np.arange(self.n_el), self.p + 1)
        g_of_sup = np.tile(np.arange(self.p + 1), self.n_el)
        edge = (self.elem_of_sup == 0) | (self.elem_of_sup == self.n_el - 1)
        self.wq_mask = edge | (g_of_sup == 0) | (g_of_sup == self.p)
        self.wq_idx = np.nonzero(self.wq_mask)[0]
        self._basis_cache = {}
        self._std = {}
        self._dwq = {}

    # ---- geometry of the 1D space ------------------------------------------------
    def supp_elems(self, i):
        """Real support of original function i: elements max(0, i-p) .. min(n_el-1, i)."""
        return max(0, i - self.p), min(self.n_el - 1, i)

    def basis_at_sup(self, U):
        key = tuple(np.asarray(U).tolist())
        if key not in self._basis_cache:
            self._basis_cache[key] = basis_all(U, self.p, self.t_sup)
        return self._basis_cache[key]

    def elems_in(self, a, b):
        mids = 0.5 * (self.xb[:-1] + self.xb[1:])
        return np.nonzero((mids > a) & (mids < b))[0]

    # ---- rule 3: WQ rule of one test function on a given layout ---------------------
    def rule(self, U, k, layout_mask, kind):
        """WQ rule of test function k of knot vector U (same element partition).

        Points Q = layout points inside supp B_k; trial set J = functions of U whose
        support overlaps supp B_k; A[j, q] = B_j(t_q) (kind '00') or B_j'(t_q) ('11');
        b_j = int B_k B_j (or int B_k' B_j') by exact (p+1)-point Gauss per element.
        If every element of supp B_k carries all p+1 Gauss points the Gauss weights
        are used directly (w_q = g_q B_k(t_q)); otherwise w = A^+ b (minimum norm).
        Returns (Q, wQ): superset indices and weights.
        """
        p = self.p
        N, dN = self.basis_at_sup(U)
        F = N if kind == "00" else dN
        a, b = U[k], U[k + p + 1]
        elems = self.elems_in(a, b)
        in_supp = np.isin(self.elem_of_sup, elems)
        Q = np.nonzero(in_supp & layout_mask)[0]
        nfun = len(U) - p - 1
        J = [j for j in range(nfun) if max(U[j], a) < min(U[j + p + 1], b)]
        G = np.nonzero(in_supp)[0]
        rhs = (self.w_sup[G] * F[k, G])[None, :] @ F[np.ix_(J, G)].T
        rhs = rhs.ravel()
        full = all(np.all(layout_mask[self.elem_of_sup == e]) for e in elems)
        if full:
            wQ = self.w_sup[Q] * F[k, Q]
        else:
            A = F[np.ix_(J, Q)]
            wQ = np.linalg.lstsq(A, rhs, rcond=1e-12)[0]
        return Q, wQ

    # ---- standard rules (Sec. 2.2 step 1) --------------------------------------------
    def std_rule(self, i, kind):
        key = (i, kind)
        if key not in self._std:
            self._std[key] = self.rule(self.U, i, self.wq_mask, kind)
        return self._std[key]

    def std_weights(self, i, kind):
        """Full-length (superset) weight vector of the standard rule of function i."""
        Q, wQ = self.std_rule(i, kind)
        w = np.zeros(len(self.t_sup))
        w[Q] = wQ
        return w

    # ---- DWQ rules (Sec. 2.2 steps 3-6) ----------------------------------------------
    def dwq_candidates(self, i):
        """Element-boundary indices b strictly inside the real support of function i:
        the artificial discontinuity sits at x_b, between elements b-1 and b."""
        e_lo, e_hi = self.supp_elems(i)
        return list(range(e_lo + 1, e_hi + 1))

    def dwq_rule(self, i, b, side, kind, force_refined=False):
        """One-sided DWQ rule of original function i with the discontinuity at x_b.

        side 0 keeps the low side (elements e_lo..b-1), side 1 the high side (b..e_hi).
        Layout = WQ points + all Gauss points of elements b-1 and b (nested points).
        If every kept element of supp B_i carries the full Gauss set, the Gauss
        weights are used directly (Sec. 2.2, last paragraph).  Otherwise: insert x_b
        p times (C^{-1}), S from knot insertion, WQ rule (rule 3) for every refined
        function on the kept side with S[i, k] != 0, and w = sum_k S[i, k] w_k.
        Returns a full-length superset weight vector (zero on the far side).
        ``force_refined`` skips the Gauss shortcut (used to pin the shortcut identity).
        """
        key = (i, b, side, kind, force_refined)
        if key in self._dwq:
            return self._dwq[key]
        p = self.p
        e_lo, e_hi = self.supp_elems(i)
        if not (e_lo < b <= e_hi):
            raise ValueError("discontinuity must lie strictly inside the support")
        xi = self.xb[b]
        layout = self.wq_mask | (self.elem_of_sup == b - 1) | (self.elem_of_sup == b)
        kept_elems = list(range(e_lo, b)) if side == 0 else list(range(b, e_hi + 1))
        w = np.zeros(len(self.t_sup))
        if not force_refined and all(np.all(layout[self.elem_of_sup == e]) for e in kept_elems):
            N, dN = self.basis_at_sup(self.U)
            F = N if kind == "00" else dN
            sel = np.isin(self.elem_of_sup, kept_elems)
            w[sel] = self.w_sup[sel] * F[i, sel]
        else:
            U_ref, S = subdivision_matrix(self.U, p, xi, p)
            lo_x, hi_x = (self.xb[e_lo], xi) if side == 0 else (xi, self.xb[e_hi + 1])
            for k in range(len(U_ref) - p - 1):
                if S[i, k] == 0.0:
                    continue
                if U_ref[k] >= lo_x and U_ref[k + p + 1] <= hi_x:
                    Q, wQ = self.rule(U_ref, k, layout, kind)
                    w[Q] += S[i, k] * wQ
        self._dwq[key] = w
        return w
