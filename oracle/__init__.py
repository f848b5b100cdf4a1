"""CPU oracle for fast WQ/DWQ formation on cut tensor-product B-spline meshes.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant with the CUDA library; the two meet only through
the seeded input descriptions in ``paper_2211_06427_gb300.synthetic`` (plain
data, none of the method's arithmetic).

Everything is plain numpy in float64, written from Marussig, "Fast formation
and assembly for spline-based 3D fictitious domain methods" (arXiv 2211.06427):

* ``bspline``   Gauss-Legendre nodes, Cox-de Boor basis values/derivatives and
                knot insertion (the 1D toolkit behind Sec. 2.2, steps 1 and 3).
* ``wq``        weighted-quadrature rules per test function (Sec. 1, the WQ
                ingredient; Sec. 2.2 step 1) and discontinuous WQ rules
                (Sec. 2.2 steps 3-6, one-sided weights, Gauss-superset layout).
* ``geometry``  level sets, cell classification with an octree for cut cells,
                function types (Sec. 2.1), the choice of the artificial
                discontinuity (Sec. 2.2 step 2) and the CSR pattern.
* ``formation`` O1: element-wise Gauss formation ("Standard Gauss (Ref)",
                Sec. 3.1) and O2: row-wise WQ/DWQ formation (Sec. 2.2, Eq. 1).
* ``adjoint``   dJ/dc for J = lambda^T A(c) u, by explicit per-point loops.
* ``sfrow``     (with ``sfrow.c``) the same O2 rows, row by row with the 3D sums taken
                one direction at a time (Table 2, row loop + sum factorization), in plain
                C on host threads; also the Hybrid Gauss and Standard Gauss variants
                (Sec. 3.1) and the load vector.  Used for large row samples and the timed
                CPU baseline; pinned against the plain loops above.

Readings of the paper where it is silent (point subset, min-norm weights, box
choice, cut-cell rule, ...) are stated in each function's docstring; the same
readings are implemented independently by the CUDA library.
"""
