"""CPU oracle for the PMCHWT (Omit) proxy fast direct solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA path (``paper_2603_09381_gb300``); the two meet
only through the seeded input descriptors of ``paper_2603_09381_gb300.workloads``
(plain numbers: shapes, centres, wavenumbers, angles).

Everything is complex128 / float64, written for readability, not speed.

Modules and the passages of the paper (arXiv 2603.09381, "An accelerated
direct solver for scalar wave scattering by multiple transmissive inclusions
in two dimensions") they follow:

  geometry   -- boundary curves and Nystrom nodes (Sec. 2.2)
  quadrature -- Kress log-split weights, trigonometric differentiation
                (the self-block quadrature of Sec. 2.2, in place of the paper's
                zeta-corrected rule)
  kernels    -- fundamental solution and its normal derivatives (Sec. 2.1,
                eqs. slp/dlp/d_slp/d_dlp)
  blocks     -- Nystrom blocks A_ij of PMCHWT (Omit) / (All) (Sec. 2.2)
  dense      -- the conventional BIEM: dense assembly + partial-pivot LU
                (Sec. 4 "conventional BIEM")
  mie        -- Mie series / multipole (Foldy-Lax) exact solutions for disks
                (independent pins, not in the paper)
  cpqr       -- column-pivoted QR and interpolative decomposition
                (Sec. 3, adaptive rank)
  tree       -- quadtree of the inclusion grid, near lists, proxy circles
                (Sec. 3, Sec. 4 near field, Sec. 4.4 Morton order)
  proxy      -- the multilevel proxy/ID fast direct solver: compression,
                compressed system (eq. compressed), recovery, top LU (Sec. 3)

Parity pins (tests/test_oracle_*.py, run with -m "not gpu"):
  quadrature : Kress weights vs the closed-form Fourier coefficients of
               ln(4 sin^2(t/2)); differentiation vs analytic derivatives.
  kernels    : scipy Hankel values (library routine) at sample points.
  blocks     : circle eigenvalues of S, D, D*, N (Bessel closed forms);
               Calderon / Green identities on stars and ellipses, for the
               self blocks and for off-diagonal blocks between two curves.
  dense      : Mie series (one disk), multipole solution (two disks, 2x2
               grid), energy balance (lossless and lossy).
  cpqr       : brute-force pivots on tiny matrices, ID error on random
               low-rank matrices.
  proxy      : agreement with the dense solve within the ID tolerance;
               one inclusion degenerates to the dense solve.
"""
