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


def test_static_scratch_larger_then_smaller_and_every_precision(sfa):
    """A larger matrix first leaves its partial sums in the shared scratch; a smaller one after
    it must still match the mesh-based reduction (each call writes every entry it reads)."""
    import torch
    rng = np.random.default_rng(4)
    big = sfa.Mesh(synthetic.desc(n_el=(12, 12, 12), p=3, ls="ball", balls=[(0.5, 0.5, 0.5, 0.42)],
                                  octree_depth=2, coef="analytic"))
    small = sfa.Mesh(synthetic.desc(n_el=(6, 7, 5), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, 0.4)],
                                    octree_depth=2, coef="analytic"))
    for prec in ("fp64", "fp32", "tf32", "tf32x3", "fp32_m64", "tf32x3_m64"):
        for m in (big, small):
            lam = torch.as_tensor(rng.standard_normal(m.n_rows), device="cuda")
            u = torch.as_tensor(rng.standard_normal(m.n_rows), device="cuda")
            vals = m.form("mass", prec)
            rowptr, colind = m.pattern()
            ref = m.bilinear(vals, lam, u, prec=prec).item()
            J = sfa.bilinear_static(rowptr, colind, vals, lam, u, prec=prec).item()
            assert abs(J - ref) <= 1e-12 * max(abs(ref), 1.0) * 10, (prec, J, ref)


def test_static_scratch_empty_and_maximum_size(sfa):
    """n_rows = 0 gives J = 0 exactly; exactly 2^20 rows is accepted (a diagonal CSR of ones
    with lambda = u = 1, so J = 2^20 exactly)."""
    import torch
    n = 1 << 20
    rowptr = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    colind = torch.arange(n, dtype=torch.int32, device="cuda")
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    J = sfa.bilinear_static(rowptr, colind, ones, ones, ones).item()
    assert J == float(n)
    J0 = sfa.bilinear_static(rowptr[:1], colind, ones, ones, ones).item()
    assert J0 == 0.0


def test_static_scratch_rejects_oversized_input(sfa):
    import torch
    lib = sfa.lib()
    n = (1 << 20) + 1
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.sfa_bilinear_static(ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), n, 0,
                                 ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                 ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == 1  # SFA_ERR_INVALID_ARG, before any kernel runs
