"""Oracle for the RSRR hot path: plain, slow, FP64, CPU only.

TEST INFRASTRUCTURE.  Only the tests, the graft entry's smoke check and the
bench's CPU-baseline / reference legs may import this package.  It shares no
code with the CUDA path (paper_1510_07522_gb300); both read their inputs from
the `workloads` generators.
"""
from .rsrr_oracle import (  # noqa: F401
    coefficients, contour_points, assemble_dense, assemble_band, band_lu, band_solve,
    dense_lu, dense_solve, sample, backward_error, truncated_basis, numerical_rank,
    project, reduced_ss, backmap, eigen_residuals, inside_contour, rsrr, moment_matrix,
    contour_rule, rectangle_split, chebyshev_reduce,
)
