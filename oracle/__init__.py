"""CPU oracle for the exponential-window frequency-domain elastodynamic BEM.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it. It shares no code with the CUDA path; the only
common module is the seeded input generator ``paper_1212_3032_gb300.inputs``,
which holds no arithmetic of the method.

Everything here is plain, slow, obviously-correct complex128 / float64 numpy,
written from the paper (Xiao, Ye, Wen, "Efficiency improvement of the
frequency-domain BEM for rapid transient elastodynamic analysis"):

* ``kernels``     fundamental solutions U, T (Sec. 2.1, Eqs. Uij, Tij, Gikj)
* ``quadrature``  element integration rules (the paper does not state them;
                  the rule is fixed here and implemented independently on the
                  GPU side)
* ``bem``         dense collocation T u = U t and boundary conditions
                  A a = b (Sec. 2.1, Eqs. Tu_Ut, Aa_b); the interior field
                  by the representation formula
* ``transforms``  DFT-MFT / IDFT-MFT, windows, damping rule (Sec. 3)
* ``solvers``     direct solve, block-Jacobi GMRES, solution extrapolation
* ``aca``         adaptive cross approximation of one admissible block, with
                  the per-component check rows the library uses
                  (Sec. 4.2, Eqs. a0, lsem, a0-solution)
* ``sweep``       the whole sequence A_k a_k = b_k, k = 0..N/2 (Eq.
                  Aa_b-sequence) and the time response

Readings of the paper used throughout (each is pinned by a test):

1. Laplace form of the radial functions: i k r -> -s r / c with
   s = eta + i k dw, so entries decay like exp(-eta r / c).
2. The P-wave terms of phi and psi carry the factor (c_s / c_p)^2.
3. In G_ikj, r_i = y_i - x_i (derivative of r with respect to the field
   point); with the literal x_i - y_i the traction kernel has the wrong sign.
4. r_i in U_ij is the unit vector r_i / r.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(closed forms, Kelvin limit, Navier residual, Hooke's-law traction,
rigid-body identity, cavity closed form, transform identities, brute force).
"""
