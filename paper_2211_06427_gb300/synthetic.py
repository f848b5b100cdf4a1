"""Seeded synthetic workload descriptions.

Plain data only (mesh sizes, degrees, level-set parameters, coefficient arrays drawn
from numpy's PCG64 generator); none of the method's arithmetic lives here.  The same
description feeds the CUDA library (through ``sfa.Mesh``) and the CPU oracle.

A description is a dict with keys
  n_el (3 ints), p, lo (3), hi (3), ls in {"ball", "balls", "gyroid", "plane", "full"},
  balls (list of (cx, cy, cz, r)), gyroid_freq, gyroid_iso, plane_pt (3), plane_n (3),
  octree_depth, coef in {"const", "analytic", "bspline"}, coef_const,
  coef_bspline (float64 array of n1*n2*n3 B-spline coefficients, index k1 + n1 (k2 + n2 k3)).
"""
import numpy as np

UNIT = dict(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0))


def desc(**kw):
    base = dict(UNIT, ls="full", balls=[], gyroid_freq=6.0, gyroid_iso=0.3,
                plane_pt=(0.0, 0.0, 0.0), plane_n=(0.0, 0.0, 1.0), octree_depth=3,
                coef="const", coef_const=1.0, coef_bspline=None)
    base.update(kw)
    base["n_el"] = tuple(int(v) for v in base["n_el"])
    return base


def lognormal_coefficients(n_el, p, seed, sigma=0.5):
    """B-spline coefficients exp(N(0, sigma^2)) on the (n_el + p)^3 mesh functions."""
    n = [ne + p for ne in n_el]
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal(n[0] * n[1] * n[2]))


def c1_ball_p2_8():
    """p=2, 8^3 elements, ball r=0.4 at the centre, c = 1 + 0.5 sin(2 pi x) cos(2 pi y) z,
    octree depth 3, mass matrix."""
    return desc(n_el=(8, 8, 8), p=2, ls="ball", balls=[(0.5, 0.5, 0.5, 0.4)], octree_depth=3,
                coef="analytic")


def c2_ball_p3_32(seed=1):
    """p=3, 32^3 elements, ball r=0.37 with a seeded centre in [0.45, 0.55]^3, analytic c."""
    centre = np.random.default_rng(seed).uniform(0.45, 0.55, 3)
    return desc(n_el=(32, 32, 32), p=3, ls="ball", balls=[(*centre, 0.37)], octree_depth=3,
                coef="analytic")


def c3_gyroid_64(p, seed=2, n_el=64):
    """Degree-p, n_el^3 gyroid sin6x cos6y + sin6y cos6z + sin6z cos6x < 0.3, log-normal
    B-spline coefficient field exp(N(0, 0.25)), octree depth 3."""
    ne = (n_el, n_el, n_el)
    return desc(n_el=ne, p=p, ls="gyroid", gyroid_freq=6.0, gyroid_iso=0.3, octree_depth=3,
                coef="bspline", coef_bspline=lognormal_coefficients(ne, p, seed))


def c3_full_64(p, seed=2, n_el=64):
    """Calibration case: the uncut cube (every row interior), same coefficient draw."""
    ne = (n_el, n_el, n_el)
    return desc(n_el=ne, p=p, ls="full", octree_depth=3,
                coef="bspline", coef_bspline=lognormal_coefficients(ne, p, seed))


def c4_adjoint(seed_lu=3, seed_fd=4):
    """p=3, 32^3 on the C2 ball, c = the log-normal draw at p=3 (35^3 coefficients);
    lambda, u ~ N(0, 1) (seed 3); 50 finite-difference indices (seed 4).
    Returns (description, lambda, u, fd_indices)."""
    d = c2_ball_p3_32()
    d["coef"] = "bspline"
    d["coef_bspline"] = lognormal_coefficients(d["n_el"], 3, seed=2)
    n = 35 ** 3
    rng = np.random.default_rng(seed_lu)
    lam = rng.standard_normal(n)
    u = rng.standard_normal(n)
    fd = np.random.default_rng(seed_fd).choice(n, 50, replace=False)
    return d, lam, u, fd


def c5_batch(seed=5, count=64):
    """`count` independent meshes: n_el ~ U{8..48}, p ~ U{2..5}, 1-8 balls with centres in
    [0.2, 0.8]^3 and radii in [0.1, 0.3], analytic coefficient."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        ne = int(rng.integers(8, 49))
        p = int(rng.integers(2, 6))
        nb = int(rng.integers(1, 9))
        balls = [(*rng.uniform(0.2, 0.8, 3), float(rng.uniform(0.1, 0.3))) for _ in range(nb)]
        out.append(desc(n_el=(ne, ne, ne), p=p, ls="balls", balls=balls, octree_depth=3,
                        coef="analytic"))
    return out


def paper_plane(p, h):
    """The paper's own geometry: [-1, 1]^3 below the plane through (0.1, 0.2, 0.3) with
    normal (0.5, -0.2, 0.9), degree p, h elements per direction."""
    return desc(n_el=(h, h, h), p=p, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), ls="plane",
                plane_pt=(0.1, 0.2, 0.3), plane_n=(0.5, -0.2, 0.9), octree_depth=3, coef="const")
