"""rsrr_band_solve_noalloc: the band LU + solves of one sampling point from device pointers,
with all scratch in the library's fixed device array.  Some callers cannot allocate device
memory (their process gives all of it to its own allocator, or the call sits in a loop that
must not allocate); this entry point serves them.  Its result must equal what rsrr_sample
computes for the same point, on two calls in a row (the scratch array is reused), and what the
oracle's own band LU and solves compute (Algorithm 2 Step 2): the same X, and the same U factor,
since both pivot by |re| + |im| with ties to the lowest row."""
import math

import numpy as np
import pytest

import workloads as w
from gpu_util import open_nep, rel_err_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def band_of_point(prob, z):
    """T(z) in general-band layout (natural order), assembled on the host in FP64."""
    import oracle
    F, _ = oracle.coefficients(prob.fns, np.array([z]))
    kl, ku = oracle.rsrr_oracle.bandwidths(prob)
    return oracle.assemble_band(prob, F[0], kl, ku), kl, ku


def test_noalloc_matches_rsrr_sample_twice(rs):
    import torch
    prob = w.config0(N=1, L=6, nx=14, ny=11)
    # the one sampling point of an N = 1 contour: theta = pi
    z0 = complex(prob.gamma.real + prob.a * math.cos(math.pi), prob.gamma.imag + prob.b * math.sin(math.pi))
    h = open_nep(rs, prob, rs.RSRR_NATURAL_ORDER)
    h.sample(prob.gamma, prob.a, prob.b, 1, prob.L, prob.U, rs.RSRR_FP64, 1e-12)
    ref = h.samples()
    h.close()
    ab, kl, ku = band_of_point(prob, z0)
    import oracle
    ab_o, ipiv_o, info_o = oracle.band_lu(ab, kl, ku)
    assert info_o == 0
    X_o = oracle.band_solve(ab_o, ipiv_o, kl, ku, prob.U)
    kv = kl + ku
    dev = torch.device("cuda")
    for _ in range(2):
        d_ab = torch.from_numpy(np.ascontiguousarray(ab.T).view(np.float64).copy()).to(dev)
        d_b = torch.from_numpy(np.ascontiguousarray(prob.U.T).view(np.float64).copy()).to(dev)
        rs.rsrr_band_solve_noalloc(prob.n, kl, ku, d_ab.data_ptr(), prob.L, d_b.data_ptr())
        torch.cuda.synchronize()
        X = d_b.cpu().numpy().view(np.complex128).reshape(prob.L, prob.n).T
        assert rel_err_cols(X, ref).max() < 1e-8
        assert rel_err_cols(X, X_o).max() < 1e-8
        # U of P A = L U: band rows 0..kv (rows <= the diagonal), element by element
        U_dev = d_ab.cpu().numpy().view(np.complex128).reshape(prob.n, -1).T[:kv + 1]
        U_orc = ab_o[:kv + 1]
        assert np.abs(U_dev - U_orc).max() <= 1e-12 * np.abs(U_orc).max()


def test_noalloc_rejects_oversized_band(rs):
    import torch
    n, kl = 60000, 120          # panel blocks alone need more than the fixed scratch
    d = torch.zeros(2, device="cuda", dtype=torch.float64)
    with pytest.raises(rs.RsrrError) as e:
        rs.rsrr_band_solve_noalloc(n, kl, kl, d.data_ptr(), 1, d.data_ptr())
    assert e.value.name == "EINVAL" and "RSRR_NOALLOC_SCRATCH_BYTES" in str(e.value)
