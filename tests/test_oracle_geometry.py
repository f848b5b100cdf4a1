"""Pins for the oracle's classification, octree domain, function types (Sec. 2.1), DWQ
box choice (Sec. 2.2 step 2) and CSR pattern, on hand-made level sets."""
import itertools

import numpy as np
import pytest

from oracle.geometry import Geometry, E_IN, E_OUT, E_CUT, E_CUT_EMPTY, F_INT, F_CUT, F_EXT


def test_plane_on_knot_plane():
    """phi = x - 0.5 on 8 elements: left elements touch phi = 0 at corners (not < 0), so
    they are cut, but their pieces fill them exactly; the domain is exactly [0, 0.5] x [0,1]^2."""
    g = Geometry(dict(n_el=(8, 4, 4), p=2, ls="plane", plane_pt=(0.5, 0, 0), plane_n=(1, 0, 0),
                      octree_depth=2))
    st = g.state.reshape(4, 4, 8)
    assert np.all(st[:, :, 4:] == E_OUT)
    assert np.all(st[:, :, :3] == E_IN)
    assert np.all(st[:, :, 3] == E_CUT)
    assert abs(g.domain_volume() - 0.5) < 1e-15
    fc = g.fclass.reshape(g.n[2], g.n[1], g.n[0])
    # function i1 supported on elements i1-2..i1: interior iff i1 <= 2; exterior iff i1-2 >= 4
    assert np.all(fc[:, :, :3] == F_INT)
    assert np.all(fc[:, :, 3:6] == F_CUT)
    assert np.all(fc[:, :, 6:] == F_EXT)


def test_small_ball_inside_one_element():
    g = Geometry(dict(n_el=(4, 4, 4), p=2, ls="ball", balls=[(0.375, 0.625, 0.375, 0.05)], octree_depth=3))
    e = g.elem_index(1, 2, 1)
    assert g.state[e] == E_CUT
    assert np.sum(g.state == E_CUT) + np.sum(g.state == E_CUT_EMPTY) == 1
    assert np.all(np.delete(g.state, e) == E_OUT)
    # functions overlapping element (1, 2, 1): i_d in [e_d, e_d + p]
    for i in range(len(g.fclass)):
        i1, i2, i3 = g.unravel_fn(i)
        touches = 1 <= i1 <= 3 and 2 <= i2 <= 4 and 1 <= i3 <= 3
        assert g.fclass[i] == (F_CUT if touches else F_EXT)
    assert 0 < g.domain_volume() < (0.125 ** 3)


def test_octree_volume_converges_to_ball():
    r = 0.3
    exact = 4.0 / 3.0 * np.pi * r ** 3
    errs = []
    for D in range(0, 5):
        g = Geometry(dict(n_el=(6, 6, 6), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, r)], octree_depth=D))
        errs.append(abs(g.domain_volume() - exact) / exact)
    assert errs[-1] < 2e-3
    assert errs[-1] < errs[1] < errs[0]


def _brute_box(g, i):
    idx = g.unravel_fn(i)
    st = g.state.reshape(g.n_el[2], g.n_el[1], g.n_el[0])
    rng = [g.supp(d, idx[d]) for d in range(3)]
    cands = []
    for d in range(3):
        for side in (0, 1):
            for b in range(rng[d][0] + 1, rng[d][1] + 1):
                r = list(rng)
                r[d] = (rng[d][0], b - 1) if side == 0 else (b, rng[d][1])
                cells = list(itertools.product(*[range(a, c + 1) for a, c in r]))
                if all(st[e3, e2, e1] == E_IN for e1, e2, e3 in cells):
                    cands.append((len(cells), d, side, b))
    return cands


@pytest.mark.parametrize("desc", [
    dict(n_el=(8, 8, 8), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, 0.4)], octree_depth=2),
    dict(n_el=(7, 9, 8), p=3, ls="plane", plane_pt=(0.1, 0.6, 0.3), plane_n=(0.5, -0.2, 0.9), octree_depth=1),
    dict(n_el=(10, 10, 10), p=4, ls="gyroid", gyroid_freq=6.0, gyroid_iso=0.3, octree_depth=1),
])
def test_box_choice_is_valid_and_maximal(desc):
    """Every chosen box is all-inside and has the largest element count among all valid
    candidates; ties resolve to smallest d, then low side, then smallest b."""
    g = Geometry(desc)
    n_box = 0
    for i in np.nonzero(g.fclass == F_CUT)[0]:
        cands = _brute_box(g, int(i))
        box = g.box(int(i))
        if not cands:
            assert box is None
            continue
        n_box += 1
        best = max(c[0] for c in cands)
        first = min((c[1], c[2], c[3]) for c in cands if c[0] == best)
        assert box == (first[0], first[2], first[1])
    assert n_box > 0


def test_pattern_definition():
    g = Geometry(dict(n_el=(6, 5, 7), p=2, ls="ball", balls=[(0.4, 0.5, 0.55, 0.33)], octree_depth=2))
    n1, n2, n3 = g.n
    p = g.p
    for i in range(n1 * n2 * n3):
        cols = g.colind[g.rowptr[i]:g.rowptr[i + 1]]
        if g.fclass[i] == F_EXT:
            assert len(cols) == 0
            continue
        i1, i2, i3 = g.unravel_fn(i)
        expect = [j1 + n1 * (j2 + n2 * j3)
                  for j3 in range(n3) for j2 in range(n2) for j1 in range(n1)
                  if abs(j1 - i1) <= p and abs(j2 - i2) <= p and abs(j3 - i3) <= p
                  and g.fclass[j1 + n1 * (j2 + n2 * j3)] != F_EXT]
        assert list(cols) == expect
