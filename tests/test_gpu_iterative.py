"""The iterative sampler (rsrr_set_band_preconditioner): only the band part of T(z_j) is factored
(an incomplete factorisation in the spirit of the paper's GMRES + ILU for systems too large to
factor), and the refinement iteration with the FP64 residual of the full T(z_j) reaches the
tolerance.  Parity with the oracle's direct (dense LU) solves and eigenvalues; a preconditioner
too weak for the iteration fails with ENOTCONVERGED."""
import numpy as np
import pytest

import oracle
import workloads as w
from gpu_util import fns_of, match, rel_err_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def natural(rs, p, band):
    h = rs.Nep(p.n, p.rowptr, p.colind, p.vals, fns_of(p), rs.RSRR_NATURAL_ORDER)
    h.set_band_preconditioner(band)
    return h


@pytest.mark.parametrize("prec", ["fp64", "c64"])
@pytest.mark.parametrize("idx,s", [(0, 20), (3, 17)])
def test_time_delay_member_banded_preconditioner(rs, prec, idx, s):
    """Time-delay member (A1 random 5 %, so the full band is ~n): factoring only the grid
    Laplacian's band (half-width s in the grid ordering) and iterating gives the direct solves."""
    p = w.config3_member(idx, s=s, N=6, L=8)
    ref, infos, _ = oracle.sample(p, dense=True)
    assert np.all(infos == 0)
    h = natural(rs, p, s)
    # refined to working accuracy: the dropped part (the delay coupling off the band) is then
    # iterated away, which a sweep count of at least one shows
    mode = (rs.RSRR_FP64 if prec == "fp64" else rs.RSRR_C64_IR) | rs.RSRR_REFINE_FULL
    tol = 1e-12 if prec == "fp64" else 1e-10
    h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, mode, tol, 30)
    info = h.info()
    assert info["dense_lu"] == 0 and info["kl"] >= s
    assert info["refine_sweeps"] >= 1
    assert h.eta().max() <= 1e-15
    assert rel_err_cols(h.samples(), ref).max() < 1e-8
    h.close()


def test_time_delay_member_eigenvalues_with_banded_preconditioner(rs):
    p = w.config3_member(2, s=12, N=32, L=8)
    ref = oracle.rsrr(p, dense=True)
    h = natural(rs, p, 12)
    h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, 30)
    h.project(1e-14)
    lam, V, res = h.solve(500, 2, 1e3, 4096, True)
    assert lam.size == ref["lam"].size > 0
    assert match(lam, ref["lam"]) < 1e-9
    h.close()


def test_weak_preconditioner_fails_cleanly(rs):
    """Diagonal only (band 0) on the gun-like NEP: the iteration does not contract, and the call
    reports ENOTCONVERGED instead of returning unconverged samples."""
    p = w.config0(N=8, L=4, nx=12, ny=12)
    h = natural(rs, p, 0)
    with pytest.raises(rs.RsrrError) as e:
        h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, rs.RSRR_FP64, 1e-10, 30)
    assert e.value.name in ("ENOTCONVERGED", "ENONFINITE")
    for band in (-2, p.n):
        with pytest.raises(rs.RsrrError) as e2:
            h.set_band_preconditioner(band)
        assert e2.value.name == "EINVAL"
    h.set_band_preconditioner(-1)  # back to the full band: the direct solve works
    h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, rs.RSRR_FP64, 1e-10, 30)
    assert h.eta().max() <= 1e-10
    h.close()
