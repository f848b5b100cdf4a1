"""Stratified row samples for the full-size parity tests (test helper, no test cases).

Strata, from the oracle's own geometry (never from the library):
  interior_regular  interior rows whose support avoids the first and last element in every
                    direction (the regular pencils of the tensor-core and register kernels);
  interior_face1    interior rows of regular (i2, i3) pencils touching a face in direction 1;
  interior_face23   interior rows touching a face in direction 2 or 3 (face pencils);
  box_d{d}_{side}   cut rows whose DWQ box is in direction d, low (0) or high (1) side;
  no_box            cut rows without a DWQ box (regular part by element Gauss points);
  cut_empty         cut rows with a cut element in their support that carries no piece.
"""
import numpy as np

from oracle.geometry import E_CUT_EMPTY, F_CUT, F_INT


def _support(g, i):
    idx = g.unravel_fn(int(i))
    return [(max(0, idx[d] - g.p), min(g.n_el[d] - 1, idx[d])) for d in range(3)]


def draw(om, sizes, seed, cut_pool=6000):
    """dict stratum -> row indices (at most sizes[stratum] each, fewer if the mesh has fewer)."""
    g = om.geo
    p = om.p
    rng = np.random.default_rng(seed)
    n1, n2, _ = g.n
    ne = g.n_el
    out = {}
    ints = np.nonzero(g.fclass == F_INT)[0]
    i1, i2, i3 = ints % n1, (ints // n1) % n2, ints // (n1 * n2)

    def reg(i, d):
        return (i - p >= 1) & (i <= ne[d] - 2)

    r23 = reg(i2, 1) & reg(i3, 2)
    pools = {"interior_regular": ints[r23 & reg(i1, 0)], "interior_face1": ints[r23 & ~reg(i1, 0)],
             "interior_face23": ints[~r23]}
    for k, pool in pools.items():
        if k in sizes and len(pool):
            out[k] = rng.choice(pool, min(sizes[k], len(pool)), replace=False)
    cuts = np.nonzero(g.fclass == F_CUT)[0]
    cand = rng.choice(cuts, min(cut_pool, len(cuts)), replace=False) if len(cuts) else cuts
    st = g.state.reshape(ne[2], ne[1], ne[0])
    bins = {}
    for i in cand:
        b = g.box(int(i))
        key = "no_box" if b is None else f"box_d{b[0]}_{b[2]}"
        bins.setdefault(key, []).append(int(i))
        (a1, b1), (a2, b2), (a3, b3) = _support(g, i)
        if np.any(st[a3:b3 + 1, a2:b2 + 1, a1:b1 + 1] == E_CUT_EMPTY):
            bins.setdefault("cut_empty", []).append(int(i))
    for k, pool in bins.items():
        if k in sizes:
            out[k] = np.asarray(pool[:sizes[k]], dtype=np.int64)
    return {k: np.asarray(v, dtype=np.int64) for k, v in out.items()}


def row_errors(vals, g, ref):
    """Relative Frobenius error per row (guarded denominator)."""
    err = {}
    for i, v in ref.items():
        gv = np.asarray(vals[g.rowptr[i]:g.rowptr[i + 1]], dtype=np.float64)
        err[i] = float(np.linalg.norm(gv - v) / max(np.linalg.norm(v), 1e-300))
    return err


def report(label, strata, err):
    """Per-stratum max and median; returns the overall max."""
    worst = 0.0
    for k, rows in strata.items():
        e = [err[int(i)] for i in rows]
        if e:
            print(f"{label} {k:17s} rows {len(e):5d}  max {max(e):.2e}  median {np.median(e):.2e}")
            worst = max(worst, max(e))
    return worst


def import_oracle_tables(m, om, p):
    """The oracle's standard and one-sided DWQ weight tables into the library."""
    for d, sp in enumerate(om.spaces):
        for which, kind in ((0, "00"), (1, "11")):
            cnt, stride = m.table_size(d, which)
            W = np.zeros((sp.n, stride))
            for i in range(sp.n):
                Q, wQ = sp.std_rule(i, kind)
                W[i, :len(Q)] = wQ
            m.import_table(d, which, W)
        for which, kind in ((2, "00"), (3, "11")):
            cnt, stride = m.table_size(d, which)
            W = np.zeros((sp.n * p * 2, stride))
            for i in range(sp.n):
                e_lo, _ = sp.supp_elems(i)
                for b in sp.dwq_candidates(i):
                    for side in (0, 1):
                        w = sp.dwq_rule(i, b, side, kind)
                        seg = w[e_lo * (p + 1): e_lo * (p + 1) + stride]
                        W[(i * p + (b - e_lo - 1)) * 2 + side, :seg.size] = seg
            m.import_table(d, which, W)
