"""FP64 CPU oracle for the hierarchical multicontinuum cell-problem solve.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference that the
GPU path is checked against. Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import it; the product path (the C-ABI
library and its Python binding) never does, and it shares no code with it.
The only common dependency is the seeded input generator ``mch_inputs``.

Every function cites the passage of the paper it follows:
  * Sec. 2, Eq. (weak_galerkin): Q1 finite elements for -div(kappa grad u).
  * Sec. 2, Eqs. (phi_avar), (phi_grad): the constrained cell problems.
  * Sec. 2, Eq. (Bs_defi): the effective coefficients.
  * Sec. 3, Eq. (phi_abstract): the energy-minimisation form.
  * Sec. 3, Eq. (PhiXiI) and Eqs. (phiXiI_all), (phi_avar_corrector),
    (phi_grad_corrector): interpolation plus correction.
  * Sec. 3.1, Eq. (defi_Sn): the nested macrogrids T_n and S_n.
  * Sec. 3.2: nested FE spaces V_n with mesh size h eta^(n-1).
  * Algorithm 1: the level loop.

Where the paper is silent or ambiguous the oracle takes these readings:
homogeneous Dirichlet conditions on the RVE boundary; the constraint
sub-blocks R_q are the P^d periods of the RVE; constraint rows whose
continuum is absent from a sub-block are dropped; centroids c_mj are taken
over the integration region R_p; effective coefficients are reported as
(1/|R_p|) int_{R_p}, with kappa in every term; each linear cell function
inherits the same-index parent function; interpolation weights are the
multilinear weights of the vertices of the enclosing T_{n-1} cell; a child's
medium on the fine grid is its level-n medium prolonged piecewise-constantly.

Parity status per function: pinned (see tests/test_oracle_pins.py) unless the
docstring says "parity unpinned".
"""
