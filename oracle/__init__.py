"""FP64 CPU oracle for the adaptive-BDDC GMRES solver of arXiv 2501.01676.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import this package.  The CUDA library never calls it and shares no code
with it: both sides are written independently from the paper's definitions
(Sect. 2-3) and meet only through the seeded input generators, which hold
none of the method's arithmetic.

Modules
-------
mesh    tensor hexahedral mesh, tensor partition, interface classification
fem     stabilised Q1 element integrals (Sect. 2), P1 on the six Kuhn
        tetrahedra of each brick (Sect. 4, Example 4.1), lifting of
        non-homogeneous Dirichlet values, global assembly, direct solve
bddc    subdomain Schur complements, deluxe scaling, face GEP, new and
        conventional edge GEPs, primal constraints, the BDDC preconditioner
        (Sect. 3)
krylov  right-preconditioned GMRES with modified Gram-Schmidt (Sect. 4)
mlp     reference forward/backward of the edge-count MLP

Parity unpinned: nothing.  Every function is pinned by a ``-m "not gpu"``
test (closed forms, invariants, brute force or library special cases).
"""
