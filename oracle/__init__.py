"""Plain FP64 CPU oracle for the FFT/Picard classical-DFT hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and nothing here imports the product.

What it computes (Knepley, Karpeev, Davidovits, Eisenberg, Gillespie,
"An Efficient Algorithm for Classical Density Functional Theory in Three
Dimensions: Ionic Solutions", arXiv:0910.1531):

* ``units``      -- physical constants, Bjerrum length, molar conversion.
* ``bulk``       -- bath thermodynamics, App. A (Percus-Yevick hard-sphere
                    chemical potential and pressure, MSA Gamma, eta, Omega and
                    the electrostatic bath chemical potential).
* ``fourier``    -- the wave-vector ordering of App. B (eq. Kvalues) and the
                    3D discrete Fourier transform written out as its defining
                    sums (one explicit DFT matrix per axis; a brute-force triple
                    sum for tiny grids).  No FFT library is used.
* ``weights``    -- analytic transforms of the FMT weights (App. B, eqs.
                    OmegaHat2, omegaHat0and1, omegaHat3, omegaHatV2), of the
                    bulk-fluid kernel (Sec. "Bulk Fluid Method", eq.
                    CplusPsiHat) and the FD-Laplacian symbol of eq.
                    potentialSolution.
* ``fmt``        -- the antisymmetrised Rosenfeld free-energy density (eq. Phi)
                    and its ten partial derivatives, with the |nV2| <= n2 bound
                    of Sec. "Numerical Stability" / App. C.
* ``functional`` -- weighted densities (eqs. nDef, conv), the hard-sphere
                    back-convolution (eq. muHS), the mean-field Poisson solve
                    (eqs. potentialSolution, potentialConstraint), the
                    bulk-fluid screening term (eq. muESexpansion), the
                    fixed-point map G (eq. rhoEquation), the grand potential
                    and its gradients.
* ``picard``     -- Picard iteration with the quadratic line search and the
                    n3 <= 0.9 step bound (Sec. "Nonlinear solver").

Parity status per function is listed in each module header.  Every function
is pinned by ``tests/test_oracle_*.py`` against closed forms, textbook limits,
quadrature of the paper's defining integrals, brute force on tiny grids or
invariants stated in the paper; none is checked only against itself.
"""
