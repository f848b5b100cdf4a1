"""The allocation-free reduction (sfa_bilinear_static) against the mesh-based sfa_bilinear.

sfa_bilinear_static exists for callers that may not allocate device memory where they
need J = lambda^T A u; its scratch is a fixed array inside the library, shared by all
calls.  This file runs last so that a failure here leaves every other test already run."""
import ctypes

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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_matches_mesh_reduction(sfa, prec):
    import torch
    desc = synthetic.desc(n_el=(10, 10, 10), p=3, ls="ball", balls=[(0.52, 0.47, 0.5, 0.36)], octree_depth=2,
                          coef="analytic")
    m = sfa.Mesh(desc)
    rng = np.random.default_rng(9)
    lam = torch.as_tensor(rng.standard_normal(m.n_rows), device="cuda")
    u = torch.as_tensor(rng.standard_normal(m.n_rows), device="cuda")
    vals = m.form("stiffness", prec)
    rowptr, colind = m.pattern()
    ref = m.bilinear(vals, lam, u, prec=prec).item()
    for _ in range(2):  # two calls in a row share (and overwrite) the same scratch
        J = sfa.bilinear_static(rowptr, colind, vals, lam, u, prec=prec).item()
        torch.cuda.synchronize()
        assert abs(J - ref) <= 1e-12 * max(abs(ref), 1.0) * 10, (J, ref)


def test_static_scratch_rejects_oversized_input(sfa):
    import torch
    lib = sfa.lib()
    n = (1 << 20) + 1
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.sfa_bilinear_static(ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), n, 0,
                                 ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                 ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == 1  # SFA_ERR_INVALID_ARG, before any kernel runs
