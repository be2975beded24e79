"""FP64 CPU oracle for the staggered finite-volume Navier-Stokes method of
Gelfgat, "Linear instability of the lid-driven flow in a cubic cavity"
(arXiv 1704.08521).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this code;
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code,
constants or helpers with the CUDA path.

Every function is a plain, slow restatement of the paper's definitions in
float64 numpy:

* ``grid``      -- stretched grids (Section 3, Eq. 5, plus the cosine map).
* ``fv``        -- staggered finite-volume residual F(U,P) of Eqs. 1-4, the
                   analytic Jacobian (Eq. 6 / Eq. 10), divergence, gradient.
* ``poisson``   -- exact Neumann pressure-correction solve by tensor-product
                   factorisation (the TPF idea of Section 3).
* ``simple``    -- the SIMPLE-like Krylov-vector algorithm of Section 3
                   (Eqs. 8-10 and the three-step loop after Eq. 10).
* ``krylov``    -- GMRES(m) and the Newton method of Section 3.
* ``arnoldi``   -- implicitly restarted Arnoldi for the eigenproblem Eq. 7.
* ``dense``     -- brute-force dense spectrum of the projected Jacobian.
* ``critical``  -- secant search for Re_cr (Section 3) and Richardson
                   extrapolation (Section 5, Table 3).

Parity status of each function is stated in its module docstring; functions
with no independent pin say "parity unpinned".
"""
