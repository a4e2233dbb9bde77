"""The complex64 band LU with tensor-core trailing updates and TMA-staged panels (Algorithm 2,
Step 2), against the oracle's band LU solves and against the CUDA-core kernels.

Bands with 32 <= kl <= 224 take this path.  The cases cover several panels and a ragged tail
(n not a multiple of 32), an odd kl (the library pads ku so the band's dense view is TMA
addressable), an unsymmetric band (kl != ku), pivoting that moves rows across the panel, the
trailing range ending inside a chunk, and a zero pivot."""
import numpy as np
import pytest
import scipy.sparse as sp

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


def run(rs, prob, precision, tol, max_refine=20, flags=0):
    h = open_nep(rs, prob, flags)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, precision, tol, max_refine)
    out = h.samples(), h.eta(), h.info()
    h.close()
    return out


def banded_problem(n, kl, ku, seed, N=6, L=5, shift=0.0):
    """T(z) = A0 - z I with A0 a random complex band matrix (kl, ku): partial pivoting moves
    nearly every row, and for kl >> ku the matrix is ill-conditioned (up to ~1e9), where only
    backward errors are comparable between solvers.  A diagonal shift makes A0 well conditioned."""
    rng = np.random.default_rng(seed)
    diags, offs = [], []
    for o in range(-kl, ku + 1):
        m = n - abs(o)
        d = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        diags.append(d + shift if o == 0 else d)
        offs.append(o)
    A0 = sp.diags(diags, offs, shape=(n, n), format="csr")
    rowptr, colind, vals = w.problems._union([A0, -sp.identity(n, format="csr")])
    return w.problems.Problem(name="band", n=n, rowptr=rowptr, colind=colind, vals=vals,
                              fns=[w.Fn(w.FN_CONST), w.Fn(w.FN_Z)], gamma=0.3 + 0.2j, a=0.5, b=0.4, N=N, L=L,
                              U=w.problems.probe_matrix(n, L, seed + 1), seed=seed)


def host_eta(prob, X):
    z, _ = oracle.contour_rule(prob.gamma, prob.a, prob.b, prob.N)
    F, _ = oracle.coefficients(prob.fns, z)
    return np.concatenate([oracle.backward_error(prob, F[j], X[:, j * prob.L:(j + 1) * prob.L], prob.U)
                           for j in range(prob.N)])


CASES = [
    ("config1", dict(s=40, N=8, L=8)),            # kl = 40: 50 panels, kv = 80 (two chunks)
    ("config1", dict(s=37, N=4, L=3)),            # kl = 37 odd, n = 1369 (ragged last panel)
    ("config1", dict(s=96, N=4, L=4)),            # kl = 96, kv = 192: chunk 0 + three 64-column chunks
    ("config0", dict(N=6, L=16, nx=40, ny=33)),   # gun-like, kl = 33, square-root terms
]


@pytest.mark.parametrize("name,kw", CASES)
def test_tc_band_lu_refined_matches_oracle(rs, name, kw):
    prob = w.by_name(name, **kw)
    X, eta, info = run(rs, prob, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10)
    assert info["band_lu_tc"] == 1 and info["dense_lu"] == 0
    ref, infos, _ = oracle.sample(prob)
    assert np.all(infos == 0)
    assert eta.max() <= 2e-15
    assert rel_err_cols(X, ref).max() < 1e-9


@pytest.mark.parametrize("n,kl,ku,seed", [(700, 48, 48, 1), (450, 33, 120, 3)])
def test_tc_band_lu_unsymmetric_bands(rs, n, kl, ku, seed):
    """Condition numbers 3e3 and 8e4 with pivoting on most rows: refined to working accuracy."""
    prob = banded_problem(n, kl, ku, seed)
    X, eta, info = run(rs, prob, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, flags=rs.RSRR_NATURAL_ORDER)
    assert info["band_lu_tc"] == 1
    assert (info["kl"], info["ku"]) == (kl, ku)
    ref, _, _ = oracle.sample(prob)
    assert eta.max() <= 2e-15
    assert rel_err_cols(X, ref).max() < 1e-9


@pytest.mark.parametrize("n,kl,ku,seed", [(1500, 36, 300, 7), (2000, 40, 600, 5), (2600, 200, 760, 6)])
def test_tc_backward_solve_wide_upper_band(rs, n, kl, ku, seed):
    """Upper bandwidths that change the backward solve's shared-memory plan: kv = 336 (a TMA ring of
    eight U12 chunk buffers), 640 and 960 (four; the band path takes ku <= 768, wider bands and
    5 (kl + ku) > 2 n go to the dense LU, so the two-buffer ring is not reached through the API).
    The diagonal shift keeps cond(T(z)) small, so the refined samples compare with the oracle's
    column by column."""
    prob = banded_problem(n, kl, ku, seed, shift=float(np.sqrt(kl + ku)))
    X, eta, info = run(rs, prob, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, flags=rs.RSRR_NATURAL_ORDER)
    assert info["band_lu_tc"] == 1
    ref, _, _ = oracle.sample(prob)
    assert eta.max() <= 2e-15
    assert rel_err_cols(X, ref).max() < 1e-9


@pytest.mark.parametrize("n,kl,ku,seed", [(613, 64, 17, 2), (1000, 224, 30, 4), (700, 48, 48, 1)])
def test_tc_band_lu_backward_error_unrefined(rs, n, kl, ku, seed):
    """One complex64 solve without refinement.  Its normwise backward error does not depend on
    the condition number (up to 2e9 here), so the tensor-core factor must give the complex64 level
    (the CUDA-core factor's, within a small factor), recomputed on the host from X."""
    prob = banded_problem(n, kl, ku, seed)
    Xt, et, it = run(rs, prob, rs.RSRR_C64_IR, 1e-2, max_refine=0, flags=rs.RSRR_NATURAL_ORDER)
    Xc, ec, ic = run(rs, prob, rs.RSRR_C64_IR, 1e-2, max_refine=0,
                     flags=rs.RSRR_NATURAL_ORDER | rs.RSRR_BAND_CUDA_CORES)
    assert it["band_lu_tc"] == 1 and ic["band_lu_tc"] == 0
    he = host_eta(prob, Xt)
    assert np.allclose(et, he, rtol=1e-6, atol=0)
    assert he.max() < 1e-5
    assert he.max() < 8 * host_eta(prob, Xc).max()


def test_tc_factor_accuracy_matches_cuda_cores(rs):
    """One unrefined complex64 solve: the tensor-core factor (BF16x3 products, FP32
    accumulation) must be as accurate as the CUDA-core FP32 factor: backward errors of the same
    order, and both within the complex64 solve's forward-error level of the FP64 oracle."""
    prob = w.config1(s=64, N=6, L=6)
    ref, _, _ = oracle.sample(prob)
    Xt, et, it = run(rs, prob, rs.RSRR_C64_IR, 1e-3, max_refine=0)
    Xc, ec, ic = run(rs, prob, rs.RSRR_C64_IR, 1e-3, max_refine=0, flags=rs.RSRR_BAND_CUDA_CORES)
    assert it["band_lu_tc"] == 1 and ic["band_lu_tc"] == 0
    assert et.max() < 4 * ec.max() + 1e-12
    assert et.max() < 1e-5
    assert rel_err_cols(Xt, ref).max() < 1e-3 and rel_err_cols(Xc, ref).max() < 1e-3


def test_tc_full_pipeline_matches_cuda_cores(rs):
    """Project and solve after the tensor-core sampling give the eigenvalues of the CUDA-core
    path (config 1b: eigenvalues inside its ellipse)."""
    prob = w.config1b(s=48, N=32, L=8)
    lams = []
    for flags in (0, rs.RSRR_BAND_CUDA_CORES):
        h = open_nep(rs, prob, flags)
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10)
        h.project(1e-14)
        lam, _, res = h.solve(500, 2, 1e3, 4096, False)
        lams.append(np.sort_complex(lam))
        h.close()
    assert lams[0].size == lams[1].size > 0
    assert np.max(np.abs(lams[0] - lams[1]) / np.abs(lams[1])) < 1e-9


def test_tc_zero_pivot_reports_singular(rs):
    """T(z) = D - z I with explicit zeros on 40 sub- and superdiagonals (so kl = ku = 40 and the
    tensor-core path runs) and d_0 equal to the first sampling point: column 0 of T(z_0) is zero."""
    import math
    n, kl, N = 200, 40, 8
    gamma, a, b = 3.0 + 1.0j, 2.0, 1.0
    t0 = 2 * math.pi * 0.5 / N
    z0 = complex(gamma.real + a * math.cos(t0), gamma.imag + b * math.sin(t0))
    d = 10.0 + np.arange(n, dtype=np.complex128)
    d[0] = z0
    rows, cols = [], []
    for o in (-kl, kl):
        r = np.arange(max(0, -o), min(n, n - o))
        rows.append(r)
        cols.append(r + o)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    Z = sp.coo_matrix((np.zeros(rows.size), (rows, cols)), shape=(n, n)).tocsr()
    # Z as a term of its own: a sum would drop its explicit zeros from the pattern
    rowptr, colind, vals = w.problems._union([sp.diags(d).tocsr(), Z, -sp.identity(n, format="csr")])
    fns = [(w.FN_CONST, [0, 0, 0, 0]), (w.FN_CONST, [0, 0, 0, 0]), (w.FN_Z, [0, 0, 0, 0])]
    h = rs.Nep(n, rowptr, colind, vals, fns, rs.RSRR_NATURAL_ORDER)
    with pytest.raises(rs.RsrrError) as e:
        h.sample(gamma, a, b, N, 2, np.ones((n, 2)), rs.RSRR_C64_IR, 1e-10)
    assert e.value.name == "ESINGULAR"
    assert h.info()["band_lu_tc"] == 1
    h.close()
