"""FP64 CPU oracle for the FreeForm subspace-construction path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code,
constants or helpers with the CUDA library in ``paper_2605_29318_gb300``; the
only module both sides use is the seeded input generator
``paper_2605_29318_gb300.synth``, which holds none of the method's arithmetic.

What it computes, in plain FP64 (citations are to the FreeForm paper):

* ``rkpm``      -- brute-force support neighbours and the corrected RKPM shape
                   functions and their gradients (Sec. 3.2, Eqs. 6-11).
* ``assembly``  -- the weight-space Hessian of Prop. 1 and the RKPM mass matrix
                   (Sec. 3.2, Eq. 14), plus the Neo-Hookean potential of
                   Eq. 16 evaluated through the deformation gradient of the
                   proof of Prop. 1 (Supp. Sec. C) for finite-difference pins.
* ``twoset``    -- the paper's own two-set discretisation (Supp. Sec. B "RKPM
                   construction"): farthest-point kernel centres chosen from
                   grid quadrature points, radii reaching two other centres,
                   Gaussian-kernel shape functions at the quadrature points
                   and the K x K H_w and M.
* ``eigen``     -- the lowest-k generalized eigenpairs of H_w c = lambda M c
                   (Sec. 3.2, Eq. 15; Supp. Sec. B "Eigenanalysis") by a dense
                   LAPACK solve, a sparse shift-invert tier, residuals and
                   M-principal angles.
* ``jacobi``    -- a hand-written cyclic Jacobi eigensolver used only to pin the
                   LAPACK call on tiny inputs.

Every function here is pinned by ``tests/test_oracle_pins.py`` (``twoset`` by
``tests/test_oracle_twoset.py``) against facts
the paper and the mathematics fix (reproducing conditions, finite differences
of the energy, invariances, brute force).  Equation numbers follow the order in
which LaTeX numbers the paper's displayed equations (Eq. 1 = the LBS map).
"""
