"""GPU adjoint dJ/dc for J = lambda^T A(c) u (c a B-spline coefficient field) against the
oracle's per-point gradient, the Euler identity (J is linear in c) and central finite
differences through the library's own forward formation."""
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


CASES = {
    "ball_p2_8": lambda: synthetic.desc(n_el=(8, 8, 8), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, 0.37)],
                                        octree_depth=2, coef="bspline",
                                        coef_bspline=synthetic.lognormal_coefficients((8, 8, 8), 2, 11)),
    "plane_p3_7x6x8": lambda: synthetic.desc(n_el=(7, 6, 8), p=3, ls="plane", plane_pt=(0.1, 0.6, 0.3),
                                             plane_n=(0.5, -0.2, 0.9), octree_depth=2, coef="bspline",
                                             coef_bspline=synthetic.lognormal_coefficients((7, 6, 8), 3, 12)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_gradient_matches_oracle(sfa, name, op):
    import torch
    from oracle.formation import OracleMesh
    from oracle import adjoint
    desc = CASES[name]()
    m = sfa.Mesh(desc)
    rng = np.random.default_rng(1)
    lam, u = rng.standard_normal(m.n_rows), rng.standard_normal(m.n_rows)
    g = m.backward(op, torch.as_tensor(lam, device="cuda"), torch.as_tensor(u, device="cuda")).cpu().numpy()
    om = OracleMesh(desc)
    ref = adjoint.gradient(om, op, lam, u)
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref)) * 10, np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    m.check_device_status()


@pytest.mark.parametrize("op", ["mass", "stiffness"])
def test_c4_euler_and_finite_differences(sfa, op):
    """C4: p=3, 32^3 ball, 35^3 cubic coefficients; central differences (h = 1e-6) on the
    50 seeded coefficients through the library's forward formation and reduction."""
    import torch
    desc, lam, u, fd_idx = synthetic.c4_adjoint()
    m = sfa.Mesh(desc)
    lam_t = torch.as_tensor(lam, device="cuda")
    u_t = torch.as_tensor(u, device="cuda")
    g = m.backward(op, lam_t, u_t).cpu().numpy()
    J = m.bilinear(m.form(op, "fp64"), lam_t, u_t).item()
    c = m.coef.cpu().numpy()
    assert abs(np.dot(c, g) - J) <= 1e-11 * (abs(J) + np.dot(np.abs(c), np.abs(g)))
    base = m.coef.clone()
    h = 1e-6
    gmax = np.max(np.abs(g))
    worst = 0.0
    for k in fd_idx:
        m.coef.copy_(base)
        m.coef[int(k)] += h
        Jp = m.bilinear(m.form(op, "fp64"), lam_t, u_t).item()
        m.coef.copy_(base)
        m.coef[int(k)] -= h
        Jm = m.bilinear(m.form(op, "fp64"), lam_t, u_t).item()
        fd = (Jp - Jm) / (2 * h)
        worst = max(worst, abs(fd - g[int(k)]))
    m.coef.copy_(base)
    # J is linear in c: the difference quotient is exact up to the rounding of J (~1e-16 |J| / h)
    assert worst <= 1e-6 * gmax, worst / gmax


def test_autograd_function(sfa):
    import torch
    desc = CASES["ball_p2_8"]()
    m = sfa.Mesh(desc)
    rng = np.random.default_rng(2)
    lam = torch.as_tensor(rng.standard_normal(m.n_rows), device="cuda")
    u = torch.as_tensor(rng.standard_normal(m.n_rows), device="cuda")
    F = sfa.SfaFormBilinear.build()
    coef = m.coef.clone().requires_grad_(True)
    J = F.apply(coef, m, "stiffness", lam, u)
    (3.0 * J).backward()
    g = m.backward("stiffness", lam, u).cpu().numpy()
    assert np.allclose(coef.grad.cpu().numpy(), 3.0 * g, rtol=1e-13, atol=1e-15 * np.max(np.abs(g)))
