"""Python side of the C row oracle (``oracle/sfrow.c``).  Test infrastructure only (see
``oracle/__init__``).

``RowOracle`` hands the numpy oracle's 1D rules and geometry to the C library, which forms
whole rows (or load values) row by row with the 3D sums evaluated one direction at a time
(the "row loop" + "sum factorization" entry of the paper's cost table for weighted
quadrature, Sec. 1, Table 2), on as many host threads as asked.  It computes what O2 of
``oracle.formation`` computes; the plain quadrature-point loops of O2 are its pin.

The C library is compiled here with the host's gcc (``build``), no CPU-specific flags.
"""
import ctypes
import os
import subprocess

import numpy as np

from .geometry import F_CUT

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sfrow.c")
LIB = os.path.join(HERE, "libsfrow.so")

VARIANTS = {"dwq": 0, "hybrid": 1, "gauss": 2}
SOURCES = {"coef": 0, "paper": 1}


def build(force=False):
    """Compile sfrow.c into oracle/libsfrow.so (skipped when up to date)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", LIB, SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("building the C row oracle failed:\n" + r.stderr)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        _lib.osf_form_rows.argtypes = [vp, ctypes.c_int, vp, i64, vp, vp, ctypes.c_int]
        _lib.osf_form_rows.restype = ctypes.c_int
        _lib.osf_load_rows.argtypes = [vp, vp, i64, vp, ctypes.c_int]
        _lib.osf_load_rows.restype = ctypes.c_int
        _lib.osf_basis.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp,
                                   ctypes.POINTER(ctypes.c_int)]
        _lib.osf_basis.restype = ctypes.c_int
    return _lib


D3 = ctypes.c_void_p * 3


class _Mesh(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int32), ("variant", ctypes.c_int32), ("coef_kind", ctypes.c_int32),
        ("src_kind", ctypes.c_int32),
        ("n_el", ctypes.c_int32 * 3), ("n", ctypes.c_int32 * 3), ("nsup", ctypes.c_int32 * 3),
        ("U", D3), ("t_sup", D3), ("w_sup", D3), ("std00", D3), ("std11", D3),
        ("dwq_id", D3), ("dwq00", D3), ("dwq11", D3),
        ("elem_state", ctypes.c_void_p), ("fclass", ctypes.c_void_p), ("box", ctypes.c_void_p),
        ("piece_ptr", ctypes.c_void_p), ("piece_box", ctypes.c_void_p),
        ("xg", ctypes.c_void_p), ("wg", ctypes.c_void_p),
        ("c0", ctypes.c_double), ("ck", ctypes.c_void_p),
        ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
    ]


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def basis_values(U, p, n_el, x):
    """(first function, values, derivatives) of the p+1 functions nonzero at x, from the C
    Cox-de Boor recursion."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    N = np.zeros(p + 1)
    dN = np.zeros(p + 1)
    first = ctypes.c_int()
    if lib().osf_basis(_ptr(U), p, n_el, float(x), _ptr(N), _ptr(dN), ctypes.byref(first)) != 0:
        raise ValueError("degree out of range")
    return first.value, N, dN


class RowOracle:
    """Rows of one ``OracleMesh`` formed by the C library.

    variant: "dwq" (the method), "hybrid" (no DWQ box: the regular part of a cut row by
    element Gauss points) or "gauss" (every row by element Gauss points: Standard Gauss).
    src (load vector only): "coef" (f = the mesh's coefficient field) or "paper"
    (f = sin(2xz) cos(3yz), the paper's target function, Sec. 3.1).
    """

    def __init__(self, om, variant="dwq", src="coef"):
        self.om = om
        g = om.geo
        p = om.p
        self.p = p
        self.variant = variant
        self._keep = []
        m = _Mesh()
        m.p = p
        m.variant = VARIANTS[variant]
        m.coef_kind = {"const": 0, "analytic": 1, "bspline": 2}[om.coef.kind]
        m.src_kind = SOURCES[src]
        m.c0 = om.coef.c0
        self.ck = np.ascontiguousarray(om.coef.ck.ravel() if om.coef.kind == "bspline" else np.zeros(1))
        m.ck = _ptr(self.ck)
        self.dwq_keys = [{} for _ in range(3)]
        self.dwq_vec = [([], []) for _ in range(3)]
        self.dwq_id = []
        for d, sp in enumerate(om.spaces):
            m.n_el[d] = sp.n_el
            m.n[d] = sp.n
            m.nsup[d] = len(sp.t_sup)
            arrs = [np.ascontiguousarray(sp.U, dtype=np.float64), np.ascontiguousarray(sp.t_sup),
                    np.ascontiguousarray(sp.w_sup),
                    np.ascontiguousarray(np.stack([sp.std_weights(i, "00") for i in range(sp.n)])),
                    np.ascontiguousarray(np.stack([sp.std_weights(i, "11") for i in range(sp.n)]))]
            self._keep += arrs
            m.U[d], m.t_sup[d], m.w_sup[d], m.std00[d], m.std11[d] = (_ptr(a) for a in arrs)
            ids = np.full(sp.n * p * 2, -1, dtype=np.int32)
            self.dwq_id.append(ids)
            m.dwq_id[d] = _ptr(ids)
        self.state = np.ascontiguousarray(g.state, dtype=np.int8)
        self.fclass = np.ascontiguousarray(g.fclass, dtype=np.int8)
        self.box = np.full(len(g.fclass), -1, dtype=np.int32)
        m.elem_state, m.fclass, m.box = _ptr(self.state), _ptr(self.fclass), _ptr(self.box)
        self._pieces(m)
        self.xg = np.ascontiguousarray(om.xg)
        self.wg = np.ascontiguousarray(om.wg)
        m.xg, m.wg = _ptr(self.xg), _ptr(self.wg)
        self.rowptr = np.ascontiguousarray(g.rowptr, dtype=np.int64)
        self.colind = np.ascontiguousarray(g.colind, dtype=np.int32)
        m.rowptr, m.colind = _ptr(self.rowptr), _ptr(self.colind)
        self.m = m
        self._boxed = set()

    def _pieces(self, m):
        """Pieces of every element as (lo, hi) boxes, ordered by element."""
        g = self.om.geo
        nE = len(g.state)
        counts = np.zeros(nE, dtype=np.int64)
        lists = []
        for e in sorted(g.pieces):
            pcs = g.pieces[e]
            counts[e] = len(pcs)
            if pcs:
                lists.append(np.asarray(pcs, dtype=np.int64))
        self.piece_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        P = np.concatenate(lists) if lists else np.zeros((0, 4), dtype=np.int64)
        box = np.zeros((len(P), 3, 2))
        sx = 2 ** (g.D + 1 - P[:, 0])
        for d in range(3):
            box[:, d, 0] = g.coord(d, P[:, 1 + d] * sx)
            box[:, d, 1] = g.coord(d, (P[:, 1 + d] + 1) * sx)
        self.piece_box = np.ascontiguousarray(box)
        m.piece_ptr, m.piece_box = _ptr(self.piece_ptr), _ptr(self.piece_box)

    def _prepare_boxes(self, rows):
        """DWQ boxes of the requested cut rows and the one-sided rules they use."""
        if self.variant != "dwq":
            return
        g = self.om.geo
        p = self.p
        changed = set()
        for i in rows:
            i = int(i)
            if i in self._boxed or g.fclass[i] != F_CUT:
                continue
            self._boxed.add(i)
            b = g.box(i)
            if b is None:
                continue
            d, bb, side = b
            self.box[i] = d | (side << 2) | (bb << 3)
            idx = g.unravel_fn(i)
            key = (idx[d], bb, side)
            if key in self.dwq_keys[d]:
                continue
            sp = self.om.spaces[d]
            self.dwq_keys[d][key] = len(self.dwq_vec[d][0])
            self.dwq_vec[d][0].append(sp.dwq_rule(idx[d], bb, side, "00"))
            self.dwq_vec[d][1].append(sp.dwq_rule(idx[d], bb, side, "11"))
            e_lo = max(0, idx[d] - p)
            self.dwq_id[d][(idx[d] * p + (bb - e_lo - 1)) * 2 + side] = self.dwq_keys[d][key]
            changed.add(d)
        for d in changed:
            a00 = np.ascontiguousarray(np.stack(self.dwq_vec[d][0]))
            a11 = np.ascontiguousarray(np.stack(self.dwq_vec[d][1]))
            self._keep += [a00, a11]
            self.m.dwq00[d], self.m.dwq11[d] = _ptr(a00), _ptr(a11)

    def rows(self, op, rows=None, threads=None):
        """Values (pattern order) of the given rows (all active rows by default) as a dict."""
        g = self.om.geo
        if rows is None:
            rows = np.nonzero(g.fclass != 0)[0]
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        self._prepare_boxes(rows)
        lens = self.rowptr[rows + 1] - self.rowptr[rows]
        off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(lens)])[:-1].astype(np.int64))
        out = np.zeros(int(lens.sum()) if len(rows) else 1)
        r = lib().osf_form_rows(ctypes.byref(self.m), 0 if op == "mass" else 1, _ptr(rows), len(rows), _ptr(off),
                                _ptr(out), int(threads or os.cpu_count() or 1))
        if r != 0:
            raise RuntimeError(f"C row oracle failed ({r})")
        return {int(i): out[o:o + n] for i, o, n in zip(rows, off, lens)}

    def load(self, rows=None, threads=None):
        """Load values b_i of the given rows (all active rows by default), as an array."""
        g = self.om.geo
        if rows is None:
            rows = np.nonzero(g.fclass != 0)[0]
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        self._prepare_boxes(rows)
        out = np.zeros(max(1, len(rows)))
        r = lib().osf_load_rows(ctypes.byref(self.m), _ptr(rows), len(rows), _ptr(out),
                                int(threads or os.cpu_count() or 1))
        if r != 0:
            raise RuntimeError(f"C row oracle failed ({r})")
        return out[:len(rows)]
