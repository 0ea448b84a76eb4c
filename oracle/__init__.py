"""FP64 CPU oracle for column-generation direct aperture optimization (DAO).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
restatement of Men, Jia & Jiang, "GPU-based ultra-fast direct aperture
optimization for online adaptive radiation therapy" (arXiv:1003.5402) against
which the CUDA path is checked.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference legs may import it; the product
package never does, and this package imports nothing from the product.

Every function cites the passage of the paper it follows (Sec. 2.1 Eqs. 1-7,
Sec. 2.2-2.3 Eq. 8 and the pricing loop, Sec. 4 Eqs. 9-10).  Readings of
passages the paper leaves open are stated where they are used.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, finite differences, adjoint identities, KKT
certificates, an independent library solver); none is "parity unpinned".
"""
from .dao import (  # noqa: F401
    VoxelTerms, voxel_terms, reoptimisation_terms, objective, gradient, curvature, csr64, dose, beamlet_prices,
    kadane_row, Pricing, price, aperture_mask, aperture_column, fluence, MasterResult,
    solve_master, CGResult, column_generation, fmo, kkt_residual, pricing_tolerance,
    aperture_value,
)
