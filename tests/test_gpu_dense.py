"""Dense-LU sampling (NEPs without a usable band, e.g. the time-delay batch whose A1 is a random
5% sparse matrix) and rsrr_sample_batch: parity with the oracle's dense LU solves, with the band
path on the same problem, and batch results equal to one-at-a-time results.

Bar as for the band path: FP64 mode backward error <= 1e-13 and the oracle's solution to the
forward-error level of two backward-stable solvers; complex64 + FP64 refinement to 1e-14 gives
the same agreement; eigenvalues match the oracle to 1e-9."""
import numpy as np
import pytest

import oracle
import workloads as w
from gpu_util import fns_of, match, open_nep, rel_err_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def run_sample(rs, prob, precision, tol, flags=0, max_refine=20):
    h = open_nep(rs, prob, flags)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, precision, tol, max_refine)
    return h, h.samples(), h.eta(), h.info()


# n = 400: panels of 64 with a 16-column tail; the first panels are taller than the
# shared-memory panel limit (factored in global memory), the last ones are staged.
@pytest.mark.parametrize("s,idx", [(20, 0), (17, 3)])
def test_delay_member_fp64_matches_oracle(rs, s, idx):
    prob = w.config3_member(idx, s=s, N=6, L=8)
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_FP64, 1e-12)
    assert info["dense_lu"] == 1
    ref, infos, _ = oracle.sample(prob, dense=True)
    assert np.all(infos == 0)
    assert eta.max() <= 1e-13
    assert rel_err_cols(X, ref).max() < 1e-8
    h.close()


@pytest.mark.parametrize("s,idx", [(20, 0), (23, 5)])
def test_delay_member_c64_refined_matches_oracle(rs, s, idx):
    prob = w.config3_member(idx, s=s, N=6, L=8)
    ref, _, _ = oracle.sample(prob, dense=True)
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_C64_IR, 1e-10)
    assert info["dense_lu"] == 1 and eta.max() <= 1e-10
    assert rel_err_cols(X, ref).max() < 1e-5
    h.close()
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_C64_IR, 1e-14)
    assert eta.max() <= 1e-14 and info["refine_sweeps"] >= 1
    assert rel_err_cols(X, ref).max() < 1e-8
    h.close()


@pytest.mark.parametrize("name,kw", [
    ("config0", dict(N=6, L=16)),              # n = 900: tall panels, 4-column tail
    ("planted_sqrt", dict(N=8, L=4)),          # n = 24 < one panel
    ("tiny_qep", dict(N=8, L=3)),              # n = 12
    ("planted_delay", dict(N=8, L=2)),         # diagonal: no interchanges at all
    ("config0", dict(N=4, L=5, nx=7, ny=5)),   # n = 35
])
@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_forced_dense_matches_band_oracle(rs, name, kw, prec):
    prob = w.by_name(name, **kw)
    ref, _, _ = oracle.sample(prob)
    mode = rs.RSRR_FP64 if prec == "fp64" else rs.RSRR_C64_IR
    h, X, eta, info = run_sample(rs, prob, mode, 1e-14 if prec == "c64" else 1e-12, flags=rs.RSRR_DENSE_LU)
    assert info["dense_lu"] == 1
    assert eta.max() <= (1e-14 if prec == "c64" else 1e-13)
    assert rel_err_cols(X, ref).max() < 1e-8
    h.close()


def test_dense_sampling_point_on_an_eigenvalue_is_singular(rs):
    import math
    import scipy.sparse as sp
    N, gamma, a, b = 8, 3.0 + 1.0j, 2.0, 1.0
    t0 = 2 * math.pi * 0.5 / N
    z0 = complex(gamma.real + a * math.cos(t0), gamma.imag + b * math.sin(t0))
    d = np.array([1.0, z0, 7.0, 9.0], dtype=np.complex128)
    rowptr, colind, vals = w.problems._union([sp.diags(d).tocsr(), -sp.identity(4, format="csr")])
    fns = [(w.FN_CONST, [0, 0, 0, 0]), (w.FN_Z, [0, 0, 0, 0])]
    h = rs.Nep(4, rowptr, colind, vals, fns, rs.RSRR_DENSE_LU)
    with pytest.raises(rs.RsrrError) as e:
        h.sample(gamma, a, b, N, 1, np.ones((4, 1)), rs.RSRR_FP64, 1e-10)
    assert e.value.name == "ESINGULAR"
    h.close()


def test_delay_member_eigenvalues_match_oracle(rs):
    prob = w.config3_member(2, s=12, N=32, L=8)
    ref = oracle.rsrr(prob, dense=True)
    h, X, eta, info = run_sample(rs, prob, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10)
    h.project(1e-14)
    lam, V, res = h.solve(500, 2, 1e3, 4096, True)
    assert lam.size == ref["lam"].size > 0
    assert match(lam, ref["lam"]) < 1e-9
    h.close()


def batch_members():
    probs = [w.config3_member(i, s=s, N=8, L=8) for i, s in [(0, 20), (1, 14), (2, 23), (3, 9)]]
    probs.append(w.config0(N=6, L=8, nx=12, ny=10))   # a banded NEP in the same call
    return probs


@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_batch_equals_one_at_a_time(rs, prec):
    mode = (rs.RSRR_FP64 if prec == "fp64" else rs.RSRR_C64_IR) | rs.RSRR_REFINE_FULL
    probs = batch_members()
    alone = []
    for p in probs:
        h, X, eta, info = run_sample(rs, p, mode, 1e-10)
        alone.append((X, info))
        h.close()
    hs = [open_nep(rs, p) for p in probs]
    rs.sample_batch(hs, [(p.gamma, p.a, p.b) for p in probs], [p.N for p in probs], [p.L for p in probs],
                    [p.U for p in probs], mode, 1e-10, 20)
    for p, h, (Xa, ia) in zip(probs, hs, alone):
        X, info = h.samples(), h.info()
        assert info["dense_lu"] == ia["dense_lu"]
        assert h.eta().max() <= 1e-10
        assert rel_err_cols(X, Xa).max() < 1e-10
        h.close()
    assert [ia["dense_lu"] for _, ia in alone] == [1, 1, 1, 0, 0]   # s = 9 (n = 81): band path


def test_batch_then_project_and_solve(rs):
    probs = [w.config3_member(i, s=s, N=32, L=8) for i, s in [(2, 12), (4, 10)]]
    hs = [open_nep(rs, p) for p in probs]
    rs.sample_batch(hs, [(p.gamma, p.a, p.b) for p in probs], [p.N for p in probs], [p.L for p in probs],
                    [p.U for p in probs], rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, 20)
    for p, h in zip(probs, hs):
        ref = oracle.rsrr(p, dense=True)
        h.project(1e-14)
        lam, V, res = h.solve(500, 2, 1e3, 4096, True)
        assert lam.size == ref["lam"].size > 0
        assert match(lam, ref["lam"]) < 1e-9
        h.close()


def test_batch_across_streams_and_repeats(rs):
    """Handles on different streams: the batch orders itself after each stream's queued work and
    every handle gets the same samples as in a one-stream batch; a repeated handle is refused."""
    import ctypes
    import torch
    probs = [w.config3_member(i, s=s, N=6, L=4) for i, s in [(0, 14), (1, 12), (2, 9)]]
    mode = rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL
    args = lambda ps: ([(p.gamma, p.a, p.b) for p in ps], [p.N for p in ps], [p.L for p in ps], [p.U for p in ps],
                       mode, 1e-10, 20)
    one = [open_nep(rs, p) for p in probs]
    rs.sample_batch(one, *args(probs))
    ref = [h.samples() for h in one]
    streams = [torch.cuda.Stream() for _ in probs]
    many = [rs.Nep(p.n, p.rowptr, p.colind, p.vals, fns_of(p), 0, ctypes.c_void_p(st.cuda_stream))
            for p, st in zip(probs, streams)]
    rs.sample_batch(many, *args(probs))
    for h, X in zip(many, ref):
        assert rel_err_cols(h.samples(), X).max() < 1e-10
        h.project(1e-14)  # each handle goes on on its own stream
    with pytest.raises(rs.RsrrError) as e:
        rs.sample_batch([one[0], one[0]], *args(probs[:1] * 2))
    assert e.value.name == "EINVAL"
    for h in one + many:
        h.close()
