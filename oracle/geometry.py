"""Oracle geometry: level sets, cells, octree pieces, function types, DWQ box, CSR pattern.
Test infrastructure only (see ``oracle/__init__``).

Sec. 2.1 defines the three function types by the measure of supp B_i intersected
with the domain; Sec. 2.2 step 2 picks, per cut function, the knot plane that
maximises the tensor-product block of interior elements; Sec. 2.2 / Sec. 3.1
integrate cut elements by sub-elements with Gauss rules.  The discrete readings:

* a cell (element or octree cell) is inside iff phi < 0 at its 8 corners and its
  centre, outside iff phi >= 0 at all 9 samples, else cut;
* cut cells are split into 8 children down to depth D; a cut leaf at depth D is
  kept whole iff phi(centre) < 0; inside cells at any level are kept whole.  The
  discrete domain Omega_h is the union of these axis-aligned boxes ("pieces");
* function i is exterior iff no element of its support has a piece (inside or
  cut with at least one piece), interior iff all its support elements are inside,
  and cut otherwise;
* box candidates for a cut function: direction d, element boundary b strictly
  inside the support in d, side low/high; the box is the full support in the
  other directions times the kept side in d; valid iff every box element is
  inside; the valid box with the most elements wins, ties broken by smallest d,
  then low side, then smallest b;
* pattern: row i is active iff i is not exterior; its columns are the active j
  with |j_d - i_d| <= p in every direction, ascending in j = j1 + n1 (j2 + n2 j3).

Sample coordinates are x(k, N) = lo + (hi - lo) * (k / N) with N = n_el * 2^(D+1),
so corners and centres of every cell up to depth D are exact grid samples.
"""
import numpy as np

OUTSIDE, INSIDE, CUT = 0, 1, 2
# element states
E_OUT, E_IN, E_CUT, E_CUT_EMPTY = 0, 1, 2, 3
# function classes
F_EXT, F_INT, F_CUT = 0, 1, 2


def _g(desc, name, default=None):
    if isinstance(desc, dict):
        return desc.get(name, default)
    return getattr(desc, name, default)


def phi_fn(desc):
    """Level-set function phi(x, y, z) (inside: phi < 0), fixed evaluation order."""
    kind = _g(desc, "ls")
    if kind == "full":
        return lambda x, y, z: np.full(np.broadcast(x, y, z).shape, -1.0)
    if kind in ("ball", "balls"):
        balls = np.asarray(_g(desc, "balls"), dtype=np.float64).reshape(-1, 4)

        def f(x, y, z):
            out = None
            for cx, cy, cz, r in balls:
                dx, dy, dz = x - cx, y - cy, z - cz
                v = np.sqrt((dx * dx + dy * dy) + dz * dz) - r
                out = v if out is None else np.minimum(out, v)
            return out
        return f
    if kind == "gyroid":
        fr = float(_g(desc, "gyroid_freq"))
        iso = float(_g(desc, "gyroid_iso"))

        def f(x, y, z):
            X, Y, Z = fr * x, fr * y, fr * z
            return ((np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z)) + np.sin(Z) * np.cos(X)) - iso
        return f
    if kind == "plane":
        p0 = np.asarray(_g(desc, "plane_pt"), dtype=np.float64)
        nn = np.asarray(_g(desc, "plane_n"), dtype=np.float64)

        def f(x, y, z):
            return (nn[0] * (x - p0[0]) + nn[1] * (y - p0[1])) + nn[2] * (z - p0[2])
        return f
    raise ValueError(f"unknown level set {kind}")


class Geometry:
    """Cell states, octree pieces, function classes, DWQ boxes and the CSR pattern."""

    def __init__(self, desc):
        self.desc = desc
        self.p = int(_g(desc, "p"))
        self.n_el = tuple(int(v) for v in _g(desc, "n_el"))
        self.n = tuple(ne + self.p for ne in self.n_el)
        self.lo = tuple(float(v) for v in _g(desc, "lo", (0.0, 0.0, 0.0)))
        self.hi = tuple(float(v) for v in _g(desc, "hi", (1.0, 1.0, 1.0)))
        self.D = int(_g(desc, "octree_depth", 3))
        self.phi = phi_fn(desc)
        self.Nk = tuple(ne * 2 ** (self.D + 1) for ne in self.n_el)
        self._element_states()
        self._function_classes()
        self._pattern()
        self._boxes = {}

    # ---- sample coordinates ------------------------------------------------------------
    def coord(self, d, k):
        k = np.asarray(k, dtype=np.float64)
        return self.lo[d] + (self.hi[d] - self.lo[d]) * (k / float(self.Nk[d]))

    def _classify(self, level, g1, g2, g3):
        """9-sample classification of level-`level` cells with global indices (g1, g2, g3)."""
        sx = 2 ** (self.D + 1 - level)
        half = sx // 2
        ks = []
        for g in (g1, g2, g3):
            g = np.asarray(g, dtype=np.int64)
            ks.append((g * sx, (g + 1) * sx, g * sx + half))
        vals = []
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    vals.append(self.phi(self.coord(0, ks[0][a]), self.coord(1, ks[1][b]),
                                         self.coord(2, ks[2][c])))
        vals.append(self.phi(self.coord(0, ks[0][2]), self.coord(1, ks[1][2]), self.coord(2, ks[2][2])))
        V = np.stack(vals)
        inside = np.all(V < 0, axis=0)
        outside = np.all(V >= 0, axis=0)
        return np.where(inside, INSIDE, np.where(outside, OUTSIDE, CUT)), V[8]

    def _element_states(self):
        n1, n2, n3 = self.n_el
        e1, e2, e3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
        e1, e2, e3 = (a.transpose(2, 1, 0).ravel() for a in (e1, e2, e3))  # e = e1 + n1(e2 + n2 e3)
        cls, _ = self._classify(0, e1, e2, e3)
        state = np.where(cls == INSIDE, E_IN, np.where(cls == OUTSIDE, E_OUT, E_CUT)).astype(np.int8)
        # octree on cut elements, level by level
        cut_ids = np.nonzero(cls == CUT)[0]
        pieces = {int(e): [] for e in cut_ids}
        cur_e = cut_ids
        cur_g = np.stack([e1[cut_ids], e2[cut_ids], e3[cut_ids]], axis=1)
        for level in range(0, self.D + 1):
            if len(cur_e) == 0:
                break
            c, centre = self._classify(level, cur_g[:, 0], cur_g[:, 1], cur_g[:, 2])
            if level == 0:
                c = np.full(len(cur_e), CUT)  # the element itself is cut by construction
            keep = (c == INSIDE) | ((c == CUT) & (level == self.D) & (centre < 0))
            for e, g in zip(cur_e[keep], cur_g[keep]):
                pieces[int(e)].append((level, int(g[0]), int(g[1]), int(g[2])))
            split = (c == CUT) & (level < self.D)
            se, sg = cur_e[split], cur_g[split]
            kids_e, kids_g = [], []
            for a in (0, 1):
                for b in (0, 1):
                    for cc in (0, 1):
                        kids_e.append(se)
                        kids_g.append(2 * sg + np.array([a, b, cc]))
            cur_e = np.concatenate(kids_e) if kids_e else np.zeros(0, np.int64)
            cur_g = np.concatenate(kids_g) if kids_g else np.zeros((0, 3), np.int64)
        for e in list(pieces):
            pieces[e].sort()
            if not pieces[e]:
                state[e] = E_CUT_EMPTY
        self.state = state
        self.pieces = pieces

    def elem_index(self, e1, e2, e3):
        return e1 + self.n_el[0] * (e2 + self.n_el[1] * e3)

    def piece_box(self, piece):
        """Axis-aligned box [(a1, b1), (a2, b2), (a3, b3)] of a piece (level, g1, g2, g3)."""
        level, *g = piece
        sx = 2 ** (self.D + 1 - level)
        return [(float(self.coord(d, g[d] * sx)), float(self.coord(d, (g[d] + 1) * sx))) for d in range(3)]

    def element_box(self, e1, e2, e3):
        sx = 2 ** (self.D + 1)
        return [(float(self.coord(d, g * sx)), float(self.coord(d, (g + 1) * sx)))
                for d, g in enumerate((e1, e2, e3))]

    def domain_volume(self):
        """Exact measure of Omega_h (sum of inside elements and pieces)."""
        vol = 0.0
        for e in np.nonzero(self.state == E_IN)[0]:
            e1, e2, e3 = self.unravel_elem(e)
            bx = self.element_box(e1, e2, e3)
            vol += np.prod([b - a for a, b in bx])
        for e, pcs in self.pieces.items():
            for pc in pcs:
                vol += np.prod([b - a for a, b in self.piece_box(pc)])
        return vol

    def unravel_elem(self, e):
        n1, n2, _ = self.n_el
        return e % n1, (e // n1) % n2, e // (n1 * n2)

    # ---- function classes (Sec. 2.1) ----------------------------------------------------
    def supp(self, d, i):
        return max(0, i - self.p), min(self.n_el[d] - 1, i)

    def _function_classes(self):
        """Classify every function by the states of its real support elements."""
        n1, n2, n3 = self.n
        p = self.p
        st = self.state.reshape(self.n_el[2], self.n_el[1], self.n_el[0])  # [e3, e2, e1]
        I3, I2, I1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
        all_in = np.ones((n3, n2, n1), dtype=bool)
        any_dom = np.zeros((n3, n2, n1), dtype=bool)
        for a3 in range(p + 1):
            for a2 in range(p + 1):
                for a1 in range(p + 1):
                    E1, E2, E3 = I1 - p + a1, I2 - p + a2, I3 - p + a3
                    ok = ((E1 >= 0) & (E1 < self.n_el[0]) & (E2 >= 0) & (E2 < self.n_el[1])
                          & (E3 >= 0) & (E3 < self.n_el[2]))
                    s = np.full((n3, n2, n1), -1, dtype=np.int8)
                    s[ok] = st[E3[ok], E2[ok], E1[ok]]
                    all_in &= (~ok) | (s == E_IN)
                    any_dom |= ok & ((s == E_IN) | (s == E_CUT))
        cls = np.where(all_in, F_INT, np.where(any_dom, F_CUT, F_EXT)).astype(np.int8)
        self.fclass = cls.ravel()  # index i = i1 + n1 (i2 + n2 i3)

    def unravel_fn(self, i):
        n1, n2, _ = self.n
        return i % n1, (i // n1) % n2, i // (n1 * n2)

    def fn_index(self, i1, i2, i3):
        return i1 + self.n[0] * (i2 + self.n[1] * i3)

    # ---- DWQ box choice (Sec. 2.2 step 2) -------------------------------------------------
    def box(self, i):
        """(d, b, side) or None for cut function i."""
        if i in self._boxes:
            return self._boxes[i]
        idx = self.unravel_fn(i)
        st = self.state.reshape(self.n_el[2], self.n_el[1], self.n_el[0])
        rng = [self.supp(d, idx[d]) for d in range(3)]
        best, best_score = None, 0
        for d in range(3):
            a, b_hi = rng[d]
            for side in (0, 1):
                for b in range(a + 1, b_hi + 1):
                    r = list(rng)
                    r[d] = (a, b - 1) if side == 0 else (b, b_hi)
                    blk = st[r[2][0]:r[2][1] + 1, r[1][0]:r[1][1] + 1, r[0][0]:r[0][1] + 1]
                    if blk.size and np.all(blk == E_IN) and blk.size > best_score:
                        best, best_score = (d, b, side), blk.size
        self._boxes[i] = best
        return best

    # ---- CSR pattern (Sec. 1 row assembly) ------------------------------------------------
    def _pattern(self):
        """CSR pattern over the full index space; inactive rows have length 0."""
        n1, n2, n3 = self.n
        p = self.p
        N = n1 * n2 * n3
        active = self.fclass != F_EXT
        offs = [(d1, d2, d3) for d3 in range(-p, p + 1) for d2 in range(-p, p + 1)
                for d1 in range(-p, p + 1)]  # ascending column order
        lengths = np.zeros(N, dtype=np.int64)
        cols = []
        chunk = 4096
        for r0 in range(0, N, chunk):
            rows = np.arange(r0, min(N, r0 + chunk))
            i1, i2, i3 = rows % n1, (rows // n1) % n2, rows // (n1 * n2)
            J = np.full((len(rows), len(offs)), -1, dtype=np.int64)
            for k, (d1, d2, d3) in enumerate(offs):
                j1, j2, j3 = i1 + d1, i2 + d2, i3 + d3
                ok = (j1 >= 0) & (j1 < n1) & (j2 >= 0) & (j2 < n2) & (j3 >= 0) & (j3 < n3)
                j = np.where(ok, j1 + n1 * (j2 + n2 * j3), 0)
                ok &= active[j]
                J[:, k] = np.where(ok, j, -1)
            J[~active[rows]] = -1
            m = J >= 0
            lengths[rows] = m.sum(axis=1)
            cols.append(J[m])
        self.rowptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        self.colind = np.concatenate(cols).astype(np.int32)
        self.active = active
