"""GPU tests of the end-to-end call with host buffers (sfa_form_host).

The call forms the matrix on the device and copies the values to the host; with cut rows it
runs them in chunks and copies the values of every finished row range while the next chunk
computes.  Its values must equal the device call's bit for bit, for every precision, with
pageable and pinned host buffers, on meshes with many, all and no cut rows, and again after
the mesh is classified anew.
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


MESHES = {
    "gyroid24_p4": lambda: synthetic.c3_gyroid_64(4, n_el=24),   # B-spline c, interior and cut rows
    "ball8_p2": synthetic.c1_ball_p2_8,                          # every active row cut
    "full12_p3": lambda: synthetic.c3_full_64(3, n_el=12),       # no cut rows
}


def _coef(desc):
    return np.ascontiguousarray(desc["coef_bspline"]) if desc["coef"] == "bspline" else None


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3_m64"])
def test_form_host_equals_device(sfa, name, prec):
    import torch
    desc = MESHES[name]()
    m = sfa.Mesh(desc)
    for op in ("stiffness", "mass"):
        dev = m.form(op, prec).cpu().numpy()
        dt = np.float64 if prec == "fp64" else np.float32
        host = np.full(dev.shape, np.nan, dtype=dt)
        m.form_host(op, prec, _coef(desc), host)
        assert np.array_equal(dev, host), (name, prec, op)
        pinned = torch.full((dev.size,), float("nan"), dtype=torch.float64 if prec == "fp64" else torch.float32).pin_memory()
        m.form_host(op, prec, _coef(desc), pinned)
        assert np.array_equal(dev, pinned.numpy()), (name, prec, op)
    m.check_device_status()


def test_form_host_after_reclassification(sfa):
    desc = MESHES["gyroid24_p4"]()
    m = sfa.Mesh(desc)
    ref = m.form("stiffness", "tf32x3_m64").cpu().numpy()
    m.build_tables()
    m.classify()
    host = np.zeros(ref.shape, dtype=np.float32)
    m.form_host("stiffness", "tf32x3_m64", _coef(desc), host)
    assert np.array_equal(ref, host)
    assert m.info["n_cut_rows"] > 8  # every chunk holds cut rows


@pytest.mark.parametrize("prec", ["fp64", "tf32x3_m64"])
def test_concurrent_stages_equal_serial_stages(sfa, prec):
    """The formation runs the coefficient grid and the interior rows on a side stream beside
    the cut-element matrices; the stage profile runs every stage one after another.  Same
    values, bit for bit."""
    desc = MESHES["gyroid24_p4"]()
    m = sfa.Mesh(desc)
    for op in ("stiffness", "mass"):
        piped = m.form(op, prec).cpu().numpy()
        serial, _ = m.form_profile(op, prec)
        assert np.array_equal(piped, serial.cpu().numpy()), (prec, op)
