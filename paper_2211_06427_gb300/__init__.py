"""GB300-native fast formation of mass/stiffness matrices on cut B-spline meshes
(weighted quadrature + sum factorisation + row assembly, with discontinuous WQ for cut
test functions and octree Gauss integration of cut cells).

``paper_2211_06427_gb300.sfa``        ctypes binding of the C ABI (include/sfa.h)
``paper_2211_06427_gb300.synthetic``  seeded synthetic workload descriptions
``paper_2211_06427_gb300.build``      nvcc build of libsfa.so for sm_103a
"""
