"""GPU parity of the tensor-core precisions (the q3, q2 and q1 contractions of the interior
rows as tcgen05 kind::tf32 or kind::f16 (BF16) MMA chains) against the CPU oracle's direct WQ formation (O2).

Stated bars, relative Frobenius error per row:
  SFA_TF32X3  <= 5e-5 (the FP32 bar: head/tail split restores about FP32 accuracy);
  SFA_TF32    <= 4e-3 (operands of each stage rounded to a 10-bit mantissa, error ~ 2^-11 per
              product and stage; measured 3.5e-4 - 1.8e-3);
  SFA_BF16    <= 1.5e-2 (operands rounded to an 8-bit mantissa, kind::f16 MMAs with FP32
              accumulation: four times the TF32 rounding).
Meshes are large enough for several regular (i2, i3) pencils and several MMA row groups
along i1, with a ragged last group; full cubes put every interior row through the kernel,
balls and the gyroid mix it with cut rows and boundary pencils.
"""
import numpy as np
import pytest

from paper_2211_06427_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = {"tf32x3": 5e-5, "tf32": 4e-3, "bf16": 1.5e-2}


@pytest.fixture(scope="module")
def sfa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_06427_gb300 import build, sfa as s
    build.build()
    return s


def _errors(vals, om, rows, op):
    g = om.geo
    ref = om.form_o2(op, rows)
    err = {}
    for i, v in ref.items():
        gv = vals[g.rowptr[i]:g.rowptr[i + 1]]
        err[i] = np.linalg.norm(gv - v) / max(np.linalg.norm(v), 1e-300)
    return err


def _pencil_rows(om, n_pencils, seed):
    """Every row of a few (i2, i3) pencils whose supports are regular in i2 and i3 (the rows the
    tensor-core kernel forms), plus a few rows of boundary pencils."""
    g = om.geo
    n1, n2, n3 = g.n
    p = om.p
    ne = g.n_el
    rng = np.random.default_rng(seed)
    reg2 = [i for i in range(n2) if i - p >= 1 and i <= ne[1] - 2]
    reg3 = [i for i in range(n3) if i - p >= 1 and i <= ne[2] - 2]
    rows = []
    for _ in range(n_pencils):
        i2, i3 = int(rng.choice(reg2)), int(rng.choice(reg3))
        rows += [i1 + n1 * (i2 + n2 * i3) for i1 in range(n1)]
    for _ in range(6):
        i2, i3 = int(rng.integers(0, min(p + 1, n2))), int(rng.integers(0, n3))
        rows.append(int(rng.integers(0, n1)) + n1 * (i2 + n2 * i3))
    return [r for r in dict.fromkeys(rows) if g.fclass[r] != 0]


@pytest.mark.parametrize("p,n_el", [(2, 12), (3, 12), (4, (16, 12, 13)), (5, 14), (6, 15)])
@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_full_cube_rows(sfa, p, n_el, op):
    from oracle.formation import OracleMesh
    ne = (n_el,) * 3 if isinstance(n_el, int) else n_el
    desc = synthetic.desc(n_el=ne, p=p, ls="full", coef="bspline",
                          coef_bspline=synthetic.lognormal_coefficients(ne, p, 21))
    m = sfa.Mesh(desc)
    om = OracleMesh(desc)
    rows = _pencil_rows(om, 2, seed=p)
    for prec in ("tf32x3", "tf32", "bf16"):
        vals = m.form(op, prec).cpu().numpy().astype(np.float64)
        err = _errors(vals, om, rows, op)
        worst = max(err.values())
        print(f"p={p} {op} {prec}: max row error {worst:.2e}, median {np.median(list(err.values())):.2e}")
        assert worst <= TOL[prec], (prec, worst)
    m.check_device_status()


@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_ball_every_row(sfa, op):
    """Every active row of a ball mesh: interior rows of regular pencils on the tensor cores,
    the rest on the CUDA cores, cut rows through DWQ and the cut-cell moments."""
    from oracle.formation import OracleMesh
    desc = synthetic.desc(n_el=(14, 13, 12), p=3, ls="ball", balls=[(0.5, 0.5, 0.5, 0.42)], octree_depth=2,
                          coef="analytic")
    m = sfa.Mesh(desc)
    om = OracleMesh(desc)
    rows = [int(i) for i in np.nonzero(om.geo.fclass != 0)[0]]
    for prec in ("tf32x3", "tf32", "bf16"):
        vals = m.form(op, prec).cpu().numpy().astype(np.float64)
        err = _errors(vals, om, rows, op)
        worst = max(err.values())
        print(f"ball p=3 {op} {prec}: max row error {worst:.2e}")
        assert worst <= TOL[prec], (prec, worst)


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
def test_c3_gyroid_p4_sampled_rows(sfa, prec):
    from oracle.formation import OracleMesh
    desc = synthetic.c3_gyroid_64(4)
    m = sfa.Mesh(desc)
    om = OracleMesh(desc)
    rows = _pencil_rows(om, 1, seed=5)
    rng = np.random.default_rng(6)
    cuts = np.nonzero(om.geo.fclass == 2)[0]
    rows += [int(i) for i in rng.choice(cuts, 10, replace=False)]
    vals = m.form("stiffness", prec).cpu().numpy().astype(np.float64)
    err = _errors(vals, om, rows, "stiffness")
    worst = max(err.values())
    print(f"C3 gyroid p=4 {prec}: max row error {worst:.2e} over {len(err)} rows")
    assert worst <= TOL[prec], worst


def test_repeated_calls_identical(sfa):
    """The persistent kernel's task split depends only on the grid: two calls agree bit for bit."""
    desc = synthetic.desc(n_el=(12, 12, 12), p=4, ls="full", coef="analytic")
    m = sfa.Mesh(desc)
    a = m.form("stiffness", "tf32x3").cpu().numpy()
    b = m.form("stiffness", "tf32x3").cpu().numpy()
    assert np.array_equal(a, b)
