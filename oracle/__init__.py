"""FP64 CPU oracle for the monolithic multilevel GDSW preconditioner and FGMRES.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the CUDA
library and its binding) never imports, links or executes anything here, and this package
shares no code with it: the only common module is the seeded input generator, which holds
none of the method's arithmetic.

Plain, slow, readable NumPy/SciPy code that follows the paper step by step:
  * fem.py     -- Q2/Q1 Taylor-Hood assembly of the Stokes saddle-point system
                  (Section 2 weak form and saddle-point equation; Section 3 Carreau law);
  * gdsw.py    -- overlapping subdomains and restrictions (Section 2.1), interface
                  entities and the monolithic GDSW coarse basis by saddle-point extension
                  (Section 2.1), coarse operator, and the multilevel recursion with the
                  nested additive preconditioner (Section 2.2, four-level equation);
  * fgmres.py  -- restarted flexible GMRES with modified Gram-Schmidt (Section 3 names
                  FGMRES as the Krylov method; its details are the textbook ones).

Parity status of each function is listed in the module headers; every function carries a
pin in tests/test_oracle_pins.py (Poiseuille closed form, one-subdomain reduction,
partition of unity, constant reproduction, extension property, brute-force dense
preconditioner, level collapse, symmetry, Carreau closed form, GMRES optimality).
"""
