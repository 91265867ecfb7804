"""CPU oracle for the direct-indirect Burton-Miller solver (FP64, plain numpy/scipy).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may use it.  It shares no code with the CUDA library under
``paper_2512_14193_gb300/`` (no kernels, constants, tables or helpers); the
only common module is ``workloads.py``, which holds seeded inputs and none of
the method's arithmetic.

Every function follows a passage of the paper (Matsumoto & Matsushima,
"Efficient LU factorization exploiting direct-indirect Burton-Miller equation
for Helmholtz transmission problems"), cited in its docstring:

* ``geometry``  - equispaced Nystrom nodes on the curve (§4, Eq. dis_mixedBM setup)
* ``operators`` - S_k, D_k, D*_k, N_k kernels (§2.2) with the 1-point
                  zeta-corrected diagonal (§4)
* ``zeta``      - the high-order zeta-corrected rule of §5.3 (order 2p + 3; p = 14 is the
                  paper's order 31), weights from the generalised Euler-Maclaurin expansion
* ``systems``   - the 3N mixed system (Eq. dis_mixedBM, Theorem thm:LU blocks)
                  and the 2N ordinary system (Eq. dis_BM)
* ``dense``     - unblocked LU with partial pivoting, the Schur path of
                  Theorem thm:LU / Corollary lem:for_ssm_RHS, the block-diagonal
                  right-hand sides of Corollary lem:block_LU, backward error
* ``mie``       - Bessel-series solution on a circle (§5.1 analytical solution)
* ``farfield``  - far-field pattern from boundary data

Pins (tests/test_oracle_*.py) tie each part to something other than itself:
mpmath and Hankel-zero values printed in Table tb:ssm_eigenvalues for the
special functions, circle closed forms and convergence rates for the
quadrature (both orders; the order-31 rule also against the eigenvalues the paper
computed with it), LAPACK for the dense LU, the Mie series and the optical theorem
for the physics.  Nothing here is "parity unpinned".
"""
from .geometry import Geometry, nodes
from .operators import hankel01, layer_operators, layer_entries
from .systems import (Params, default_params, mixed_blocks, mixed_matrix, ordinary_matrix, incident, rhs_plane_wave,
                      mixed_rows, ordinary_rows)
from .dense import (lu_factor, lu_solve, dense_solve, schur_solve, block_rhs_solve, mixed_residual,
                    backward_error_mixed, backward_error_dense)
from .mie import mie_coefficients, mie_boundary, mie_far_field
from .farfield import far_field

__all__ = [
    "Geometry", "nodes", "hankel01", "layer_operators", "layer_entries", "Params", "default_params",
    "mixed_blocks", "mixed_matrix", "ordinary_matrix", "mixed_rows", "ordinary_rows", "incident", "rhs_plane_wave",
    "lu_factor",
    "lu_solve", "dense_solve", "schur_solve", "block_rhs_solve", "mixed_residual", "backward_error_mixed",
    "backward_error_dense", "mie_coefficients", "mie_boundary", "mie_far_field", "far_field",
]
