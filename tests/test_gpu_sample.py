"""Parity of rsrr_sample (Algorithm 2 Steps 1-2, Eq. eq-hatS) with the oracle's band LU solves.

Bar: FP64 mode reaches backward error <= 1e-13 per column and agrees with the oracle to the
forward-error level of two backward-stable solvers; complex64 + FP64 refinement reaches the
requested eta and the same agreement once refined to 1e-14."""
import numpy as np
import pytest

import oracle
import workloads as w
from gpu_util import open_nep, rel_err_cols, scrambled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def run_sample(rs, prob, precision, tol, max_refine=12, flags=0):
    h = open_nep(rs, prob, flags)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, precision, tol, max_refine)
    return h, h.samples(), h.eta(), h.info()


CASES = [
    ("config0", dict(N=8, L=16)),              # band 30, several panels + ragged tail
    ("config0", dict(N=4, L=5, nx=7, ny=5)),   # n = 35: one full panel + 3-row tail
    ("tiny_qep", dict(N=8, L=3)),              # n = 12 < panel width
    ("planted_delay", dict(N=8, L=2)),         # diagonal: kl = ku = 0
    ("planted_sqrt", dict(N=8, L=4)),          # banded orthogonal similarity
    ("loaded_string", dict(n=700, N=6, L=1)),  # tridiagonal, rational term, L = 1
]


@pytest.mark.parametrize("name,kw", CASES)
def test_fp64_samples_match_oracle(rs, name, kw):
    prob = w.by_name(name, **kw)
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_FP64, 1e-12)
    ref, infos, eta_ref = oracle.sample(prob)
    assert np.all(infos == 0)
    assert eta.max() <= 1e-13
    assert info["refine_sweeps"] == 0
    # both solvers are backward stable: forward differences stay at cond * u
    assert rel_err_cols(X, ref).max() < 1e-8
    h.close()


@pytest.mark.parametrize("name,kw", [("config0", dict(N=8, L=16)), ("config1", dict(s=24, N=8, L=8)),
                                     ("planted_sqrt", dict(N=8, L=4))])
def test_c64_refined_samples_match_oracle(rs, name, kw):
    prob = w.by_name(name, **kw)
    ref, _, _ = oracle.sample(prob)
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_C64_IR, 1e-10)
    assert eta.max() <= 1e-10
    assert rel_err_cols(X, ref).max() < 1e-5
    h.close()
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_C64_IR, 1e-14)
    assert eta.max() <= 1e-14
    assert info["refine_sweeps"] >= 1
    assert rel_err_cols(X, ref).max() < 1e-8
    h.close()


def test_reordering_is_invisible(rs):
    prob = w.config0(N=4, L=4, nx=10, ny=8)
    sc, p = scrambled(prob)
    h, X, eta, info = run_sample(rs, sc, rs.RSRR_FP64, 1e-12)
    assert info["natural_order"] == 0
    assert max(info["kl"], info["ku"]) <= 12          # RCM finds a narrow band again
    ref, _, _ = oracle.sample(prob)
    assert rel_err_cols(X, ref[p]).max() < 1e-8       # results come back in the caller's order
    h.close()
    h, X2, _, info2 = run_sample(rs, sc, rs.RSRR_FP64, 1e-12, flags=rs.RSRR_NATURAL_ORDER)
    assert info2["natural_order"] == 1 and info2["kl"] > 40
    assert rel_err_cols(X2, ref[p]).max() < 1e-8
    h.close()


def test_reuse_resident_probe_matrix(rs):
    prob = w.config0(N=4, L=4, nx=9, ny=9)
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12)
    X1 = h.samples()
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, None, rs.RSRR_FP64, 1e-12)
    assert np.array_equal(X1, h.samples())
    with pytest.raises(rs.RsrrError) as e:
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L + 1, None, rs.RSRR_FP64, 1e-12)
    assert e.value.name == "EINVAL"
    h.close()


def test_sampling_point_on_an_eigenvalue_is_singular(rs):
    import math
    import scipy.sparse as sp
    N, gamma, a, b = 8, 3.0 + 1.0j, 2.0, 1.0
    t0 = 2 * math.pi * 0.5 / N
    z0 = complex(gamma.real + a * math.cos(t0), gamma.imag + b * math.sin(t0))
    d = np.array([1.0, z0, 7.0, 9.0], dtype=np.complex128)
    rowptr, colind, vals = w.problems._union([sp.diags(d).tocsr(), -sp.identity(4, format="csr")])
    fns = [(w.FN_CONST, [0, 0, 0, 0]), (w.FN_Z, [0, 0, 0, 0])]
    h = rs.Nep(4, rowptr, colind, vals, fns)
    with pytest.raises(rs.RsrrError) as e:
        h.sample(gamma, a, b, N, 1, np.ones((4, 1)), rs.RSRR_FP64, 1e-10)
    assert e.value.name == "ESINGULAR"
    with pytest.raises(rs.RsrrError) as e:
        h.project(1e-14)
    assert e.value.name == "EORDER"
    h.close()


def test_refine_full_reaches_working_accuracy(rs):
    prob = w.config1(s=24, N=8, L=8)
    ref, _, _ = oracle.sample(prob)
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, 20)
    assert eta.max() <= 2e-15            # refined past tol, to FP64 working accuracy
    assert rel_err_cols(X, ref).max() < 1e-9
    h.close()


def test_unreachable_tolerance_reports_not_converged(rs):
    prob = w.config0(N=4, L=4, nx=9, ny=9)
    h = open_nep(rs, prob)
    with pytest.raises(rs.RsrrError) as e:
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_C64_IR, 1e-30, 3)
    assert e.value.name == "ENOTCONVERGED"
    h.close()
