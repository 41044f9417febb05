"""FP64 CPU oracle for the Galerkin contracting integral-equation solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library; the only
module both sides use is ``workloads`` (seeded inputs, no method arithmetic).

What it computes, each step in the paper's order and notation (Kruglyakov &
Bloshanskaya, "High-performance parallel solver for integral equations of
electromagnetics based on Galerkin method"):

* ``layered``      -- fundamental functions U_1, U_sigma of the layered medium,
                      Appendix B: eq. (lmff), recursions (pq_req), amplitudes
                      (A_rs), the overflow-free form (UU2), and the vertical
                      integrals V1..V5 of eq. (Ver_Int), integrated analytically.
* ``lateral``      -- the four-fold lateral cell-to-cell integrals of J0 in
                      eq. (Hor_Int) and their lateral derivatives, as functions
                      of lambda (Appendix C, eq. (transf)).
* ``static``       -- closed-form box-to-box integrals of 1/r used to take the
                      quasi-static singular part of touching cells out of the
                      lambda integral (a reading of Appendix C, whose filter
                      output functions are not printed).
* ``coefficients`` -- the 3x3 blocks B_n^m of Appendix A assembled into the
                      compressed tensor Q(i, j) of eq. (matrix_symm).
* ``normal``       -- the MT plane-wave normal field E^N and U^0 of (slae_matricies).
* ``operator``     -- A = S + R1 B R2 (eq. (matrix_convolv)): dense apply, FFT
                      apply (Sect. 3.3), GMRES(m) and dense LU solves, and the
                      in-cell field E = U / a (eq. (iEH320op)).
* ``proxy``        -- full-size synthetic operators (seeded random coefficients
                      scaled to make GMRES converge) whose GPU solutions the FFT
                      apply checks by their residual.

Parity status of each function is stated in its module header.
"""
