"""Parity of rsrr_sample with the oracle at the benchmark workloads' full sizes and band widths,
and the device's backward errors recomputed on the host.

Algorithm 2 Step 2 (Eq. eq-hatS) at:
  * the damped QEP on a 200 x 200 grid (n = 40000, kl = ku = 200, N = 64, L = 32): the
    benchmark workload, in the launch configuration the bench times (all 64 points in one
    factor launch, complex64 LU + FP64 refinement to working accuracy), and in plain FP64;
  * the gun-like square-root NEP on a 400 x 250 grid (n = 100000, kl = ku = 250, N = 64,
    L = 48), in both precisions.
The oracle factors only a few sampled points (its band LU takes seconds per point at these
sizes); the GPU runs every point and the sampled column blocks are compared element by element.

The metric accepts a sample at eta <= 1e-10 (the normwise backward error of reading C5), and
that eta comes from the device.  Here it is recomputed on the host from the returned X with the
oracle's pinned backward_error, column by column."""
import numpy as np
import pytest

import oracle
import workloads as w
from gpu_util import open_nep, rel_err_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def host_eta(prob, X, j):
    """eta of the L columns of point j's block, from the oracle (Frow = f_i(z_j))."""
    z, _ = oracle.contour_rule(prob.gamma, prob.a, prob.b, prob.N)
    F, _ = oracle.coefficients(prob.fns, z)
    return oracle.backward_error(prob, F[j], X, prob.U)


def test_device_eta_equals_host_eta_unrefined_c64(rs):
    """Complex64 solves without refinement leave eta near 1e-7, far above FP64 rounding of the
    residual, so the device's and the host's eta must agree to many digits per column."""
    prob = w.config1(s=40, N=8, L=6)
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_C64_IR, 1e-3, 0)
    X, eta = h.samples(), h.eta()
    assert h.info()["refine_sweeps"] == 0
    assert eta.min() > 1e-12                      # not at the rounding floor: a sharp comparison
    for j in range(prob.N):
        he = host_eta(prob, X[:, j * prob.L:(j + 1) * prob.L], j)
        assert np.allclose(eta[j * prob.L:(j + 1) * prob.L], he, rtol=1e-8, atol=0), j
    h.close()


def test_device_eta_equals_host_eta_refined(rs):
    """After refinement both sides sit at the FP64 rounding level of the residual: they must both
    certify eta <= tol, and agree within that rounding level."""
    prob = w.config0(N=8, L=8)
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, 20)
    X, eta = h.samples(), h.eta()
    for j in range(prob.N):
        he = host_eta(prob, X[:, j * prob.L:(j + 1) * prob.L], j)
        assert he.max() <= 1e-14
        assert np.all(np.abs(eta[j * prob.L:(j + 1) * prob.L] - he) <= 4e-16 + 1e-3 * he), j
    h.close()


FULL = [
    # (generator, kwargs, sampled points, (precision flags, tol, max_refine))
    ("config1", dict(), [0, 37, 63], "c64"),
    ("config1", dict(), [5, 50], "fp64"),
    ("config2", dict(), [0, 41], "c64"),
    ("config2", dict(), [20], "fp64"),
]


@pytest.mark.parametrize("name,kw,pts,prec", FULL)
def test_full_size_samples_match_oracle(rs, name, kw, pts, prec):
    prob = w.by_name(name, **kw)
    h = open_nep(rs, prob)
    if prec == "c64":
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, 20)
    else:
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-10)
    info = h.info()
    assert (info["kl"], info["ku"]) == ((200, 200) if name == "config1" else (250, 250))
    assert info["dense_lu"] == 0
    eta = h.eta()
    assert eta.max() <= 1e-10
    ref, infos, _ = oracle.sample(prob, points=pts)
    assert np.all(infos == 0)
    for k, j in enumerate(pts):
        X = h.samples(j, j + 1)
        Y = ref[:, k * prob.L:(k + 1) * prob.L]
        assert rel_err_cols(X, Y).max() < 1e-8, (j, rel_err_cols(X, Y).max())
        he = host_eta(prob, X, j)
        assert he.max() <= (2e-15 if prec == "c64" else 1e-13), (j, he.max())
    h.close()
