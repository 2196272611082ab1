"""FP64 CPU oracle for the BBWADG acoustic and elastic RK stages (test infrastructure).

This package is test infrastructure, not part of the product. Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it. It shares no code with the GPU
path: every operator here is built from its plain definition (Dirichlet
moment integrals, dense LU solves, brute-force node matching) rather than from
the sparse/telescoped forms the CUDA kernels use.

Modules
-------
bernstein   reference-tetrahedron Bernstein algebra (Sec. 2, Sec. 4, Sec. 5)
quadrature  collapsed-coordinate Gauss rules on the tetrahedron (Sec. 3.3)
mesh        connectivity, geometry and face-node matching (Sec. 3.1, Sec. 4)
acoustic    semi-discrete WADG right-hand side, LSRK stage, energy (Eq. 2, 4)
elastic     velocity-stress WADG right-hand side with the matrix weight (Sec. 2.2)
adjoint     receiver-misfit gradient by the transposed stage operators
"""
