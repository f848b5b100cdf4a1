"""GPU tests of the batched formation (one CUDA graph over many meshes) and of the
interior-tile autotuner.

A batch runs the same kernels on the same inputs as single-mesh calls, so its values must
equal them bit for bit; the single-mesh path is itself held to the oracle by the parity
tests, and one mesh of the batch is checked against the oracle here as well.
"""
import numpy as np
import pytest

from paper_2211_06427_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_06427_gb300 import build, sfa as s
    build.build()
    return s


def _small_batch(count=7, seed=15):
    """C5-style meshes (union of balls, analytic c), degrees 2..5, 6..14 elements per side."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        ne = int(rng.integers(6, 15))
        p = 2 + k % 4
        nb = int(rng.integers(1, 4))
        balls = [(*rng.uniform(0.3, 0.7, 3), float(rng.uniform(0.2, 0.35))) for _ in range(nb)]
        out.append(synthetic.desc(n_el=(ne, ne + 1, ne), p=p, ls="balls", balls=balls, octree_depth=2,
                                  coef="analytic"))
    return out


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "fp64"])
@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_batch_equals_single_calls(sfa, prec, op):
    meshes = [sfa.Mesh(d) for d in _small_batch()]
    ref = [m.form(op, prec).cpu().numpy() for m in meshes]
    got = sfa.form_batched(meshes, op, prec)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g.cpu().numpy())
    # replay of the cached graph into the same buffers
    for g in got:
        g.zero_()
    got2 = sfa.form_batched(meshes, op, prec, outs=[g.data for g in got])
    for r, g in zip(ref, got2):
        assert np.array_equal(r, g.cpu().numpy())
    for m in meshes:
        m.check_device_status()


def test_batch_tracks_reclassification(sfa):
    """A captured batch is invalidated when one of its meshes is rebuilt: the values follow."""
    meshes = [sfa.Mesh(d) for d in _small_batch(4, seed=3)]
    first = [g.cpu().numpy() for g in sfa.form_batched(meshes, "stiffness", "fp32")]
    meshes[1].build_tables()
    meshes[1].classify()
    second = [g.cpu().numpy() for g in sfa.form_batched(meshes, "stiffness", "fp32")]
    for a, b in zip(first, second):
        assert np.array_equal(a, b)


def test_batch_member_matches_oracle(sfa):
    from oracle.formation import OracleMesh
    descs = _small_batch(5, seed=8)
    meshes = [sfa.Mesh(d) for d in descs]
    vals = sfa.form_batched(meshes, "stiffness", "fp64")
    k = 2
    om = OracleMesh(descs[k])
    g = om.geo
    rng = np.random.default_rng(0)
    rows = [int(i) for i in rng.choice(np.nonzero(g.active)[0], 40, replace=False)]
    ref = om.form_o2("stiffness", rows)
    v = vals[k].cpu().numpy()
    for i, r in ref.items():
        gv = v[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.linalg.norm(gv - r) <= 1e-12 * max(np.linalg.norm(r), 1e-300)


def test_batch_rejects_bad_arguments(sfa):
    meshes = [sfa.Mesh(d) for d in _small_batch(2, seed=4)]
    with pytest.raises(sfa.SfaError):
        sfa.form_batched([meshes[0], meshes[0]], "mass", "fp32")


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_autotune_keeps_values(sfa, prec):
    """The tuned tile changes the schedule, not the arithmetic of each row."""
    desc = synthetic.desc(n_el=(20, 18, 19), p=3, ls="ball", balls=[(0.5, 0.5, 0.5, 0.45)], octree_depth=2,
                          coef="analytic")
    m = sfa.Mesh(desc)
    before = m.form("stiffness", prec).cpu().numpy()
    tuned = m.autotune("stiffness", prec).cpu().numpy()
    after = m.form("stiffness", prec).cpu().numpy()
    choice = sfa.get_tuning(3, "stiffness", prec)
    assert any(c > 0 for c in choice), choice
    assert np.array_equal(tuned, after)
    # a different chunk length regroups the shared q3/q2 stages: rounding may move by an ulp
    scale = np.max(np.abs(before))
    assert np.max(np.abs(after - before)) <= 1e-6 * scale
