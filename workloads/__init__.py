"""Seeded synthetic NEP workloads shared by the oracle and the CUDA path.

This package only *describes* problems: coefficient matrices A_i in one union
CSR pattern, the kinds and parameters of the scalar functions f_i, the contour,
the sampling sizes N and L, and the probing matrix U.  It evaluates none of the
method's arithmetic (no f_i(z), no assembly, no factorisation), so the oracle
and the CUDA path can both read it without sharing any computation.
"""
from .problems import (  # noqa: F401
    Fn, FN_CONST, FN_Z, FN_Z2, FN_ISQRT_SHIFT, FN_EXP_DELAY, FN_RATIONAL, FN_CHEBYSHEV,
    Problem, probe_matrix, grid_laplacian, config0, config0_linear, config0_rect, config1,
    config1b, config2, config3_member, config3_batch, planted_sqrt,
    planted_delay, tiny_qep, loaded_string, acoustic_1d, by_name, TzProblem, distributed_delay,
)
