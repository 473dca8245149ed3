"""CPU oracle for the domain wall fermion hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 numpy restatement of what the CUDA library computes.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library never does, and this package never
imports the library.  The two share nothing but the seeded input generators
(``paper_2203_17119_gb300.inputs``), which hold no operator arithmetic.

Modules:

* ``oracle.dwf``      -- gamma matrices, Wilson hop, Shamir/Moebius 5D
  operator and its adjoint, even-odd blocks, closed-form M_ee^-1, Schur
  operator M_pc, CGNE solve, Dirichlet block operator D_Omega (mask form and
  cut-link form), per-site evaluation for sampled checks.
* ``oracle.dense``    -- dense matrices of the above on tiny lattices, for
  brute-force inverses, determinants and the block identities of Sec. 2.1.
* ``oracle.multishift`` -- multi-shift CG for the rational functions of the
  normal operators (Sec. 2.3.1).
* ``oracle.force``    -- the link derivative of Re <X, D Y>, the insertion
  of delta D that the DD-HMC forces of Sec. 2.3 are built from, and the
  dense boundary-action and Hasenbusch-ratio forces.
* ``oracle.boundary`` -- matrix-free P, R^-1 and the boundary-action force
  for lattices too large for dense matrices.
* ``oracle.chebyshev`` -- the Chebyshev filter T_n(z(A)) v of Sec. 4.
* ``oracle.rational`` -- Zolotarev's optimal rational approximation of
  1/sqrt(x) in partial fractions.
* ``oracle.nn``       -- the parallel-transport convolutional preconditioner
  (forward, analytic backward, Adam).

Parity pins (what fixes each function independently of its own code) are in
``tests/test_oracle_*.py``.
"""
