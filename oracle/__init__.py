"""FP64 CPU oracle for the partial Fourier transform and PIE.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package. The GPU library never calls it and shares no
code, tables or constants with it; the only common module is the seeded input
generator ``paper_2408_03532_gb300.synth``.

Every function follows a passage of the paper (Parada, Wu Fung, Osher,
"Fast Partial Fourier Transforms for Large-Scale Ptychography"):

* ``coeffs``  -- Section 3.1.1 (minimax polynomial, scope xi(eps, r)),
                 Algorithm 1 and Algorithm 4 (offline tables B, W);
* ``dft``     -- the DFT definition of Section 3.1.1 and its 2-D form in
                 Appendix A, restricted to the lowest M x M frequencies;
* ``pft``     -- Algorithm 2 (1-D online PFT), Algorithm 5 (2-D online PFT)
                 and the adjoint of Algorithm 5;
* ``pie``     -- Section 2.1 (modulus projection, objective, PIE update),
                 Algorithm 3 (hybrid warm start) and the stopping rule and
                 relative error of Section 4;
* ``grad``    -- the amplitude loss and its gradient with respect to the object
                 and the probe (Section 1: differentiating through the PFT).

Pins (tests marked ``not gpu``) tie each function to something other than
itself: brute-force sums, closed forms, Parseval, the adjoint identity, the
error bound implied by Section 3.1.1, the paper's printed r = 13 at
eps = 1e-7, and noise-free recovery.
"""
