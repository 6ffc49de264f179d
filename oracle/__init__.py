"""CPU oracle for the Sakurai-Sugiura complex-band-structure method (test infrastructure).

This package is a plain, slow, FP64 restatement of what the paper computes, written
to check the CUDA library against.  It is test infrastructure only: the product
path never imports it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA path; the
only shared module is the seeded input generator (``paper_1709_09347_gb300.synth``),
which holds none of the method's arithmetic.

Modules and the passages they follow (Iwase et al., SC17, arXiv 1709.09347):

* ``fd``        central finite-difference weights of the Laplacian (§4: nine-point
                FD), solved from the Taylor conditions in exact rationals.
* ``operator``  the cell Hamiltonian blocks H_{n,n} (H0), H_{n,n+1} (H+), H_{n,n-1}
                (H-) of Eq. (2), the QEP matrix P(z) of Eq. (4), Frobenius norms.
* ``contour``   the two-circle quadrature of §3.2 (points, angles, weights).
* ``bicg``      BiCG for the systems of Eq. (9) and their duals Eq. (11) (§3.2).
* ``ss``        Algorithm 1 (moments, block Hankel, SVD cut, reduced eigenproblem),
                the residual check, the annulus filter of Eq. (5) and k = -i ln(λ)/a.
* ``dense``     brute-force companion linearisation of the QEP for tiny cells.

Every function pinned by the ``-m "not gpu"`` tests; see each module's header for its
pins.  None is "parity unpinned".
"""
