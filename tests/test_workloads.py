"""The seeded input recipes: shapes, structure and distributions of the synthetic workloads that
stand in for the paper's examples (no GPU).  Both the oracle and the CUDA path read these inputs,
so each stated property is checked on the generated arrays themselves."""
import numpy as np
import pytest

import workloads as w
from workloads import problems as wp


def semi_bandwidth(p):
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    return int(np.abs(rows - p.colind).max())


def test_probe_matrix_is_seeded_complex_gaussian():
    U = wp.probe_matrix(20000, 4, seed=3)
    assert U.shape == (20000, 4) and U.dtype == np.complex128 and U.flags.f_contiguous
    assert np.array_equal(U, wp.probe_matrix(20000, 4, seed=3))
    assert not np.array_equal(U, wp.probe_matrix(20000, 4, seed=4))
    # re and im iid N(0, 1/2): E|u|^2 = 1, mean 0, re and im uncorrelated (80000 samples)
    assert abs(np.mean(np.abs(U) ** 2) - 1.0) < 0.02
    assert abs(U.mean()) < 0.02
    assert abs(np.mean(U.real * U.imag)) < 0.01
    assert abs(np.var(U.real) - 0.5) < 0.01 and abs(np.var(U.imag) - 0.5) < 0.01


def test_gun_like_config0_recipe():
    p = w.config0()
    nx = ny = 30
    assert (p.n, p.J, p.N, p.L) == (nx * ny, 4, 32, 16)
    assert (p.gamma, p.a, p.b) == (250.0, 150.0, 150.0)
    assert semi_bandwidth(p) == ny
    K, mM, W1, W2 = (p.term(i).toarray() for i in range(4))
    assert np.allclose(K, K.T) and np.allclose(mM, -np.eye(p.n))
    h = 1.0 / (nx + 1)
    assert np.allclose(np.diag(K), 4.0 / h ** 2)
    # W1 / W2 mask the nodes with ix = 0 / ix = nx - 1 (index ix * ny + iy)
    assert np.array_equal(np.diag(W1.real), (np.arange(p.n) // ny == 0).astype(float))
    assert np.array_equal(np.diag(W2.real), (np.arange(p.n) // ny == nx - 1).astype(float))
    assert [f.kind for f in p.fns] == [wp.FN_CONST, wp.FN_Z, wp.FN_ISQRT_SHIFT, wp.FN_ISQRT_SHIFT]
    assert p.fns[2].params()[:2] == [0.0, 0.0] and p.fns[3].params()[:2] == [108.8 ** 2, 1.0]


def test_damped_qep_config1_recipe():
    p = w.config1()
    assert (p.n, p.J, p.N, p.L) == (40000, 3, 64, 32)
    assert (p.gamma, p.a, p.b) == (-0.5 + 40j, 2.0, 30.0)
    assert semi_bandwidth(p) == 200
    K, C, M = p.vals
    # Rayleigh damping C = 0.05 K + 0.02 M on the union pattern; M diagonal with entries in [1, 1.1)
    assert np.allclose(C, 0.05 * K + 0.02 * M, rtol=0, atol=1e-12 * np.abs(K).max())
    Md = p.term(2).diagonal().real
    assert Md.min() >= 1.0 and Md.max() < 1.1 and p.term(2).count_nonzero() == p.n
    assert [f.kind for f in p.fns] == [wp.FN_CONST, wp.FN_Z, wp.FN_Z2]
    assert np.array_equal(p.U, w.config1().U)


def test_gun_like_config2_recipe():
    p = w.config2()
    assert (p.n, p.J, p.N, p.L) == (400 * 250, 4, 64, 48)
    assert (p.gamma, p.a, p.b) == (330.0, 300.0, 300.0)
    assert semi_bandwidth(p) == 250
    # the branch point z = 0 of the sigma1 = 0 term stays outside the circle
    assert abs(0.0 - p.gamma) > p.a


@pytest.mark.parametrize("idx", [0, 5, 17])
def test_time_delay_member_recipe(idx):
    p = w.config3_member(idx, s=14)
    n = 14 * 14
    assert p.n == n and p.J == 3
    mI, A0, A1 = (p.term(i).toarray().real for i in range(3))
    assert np.allclose(mI, -np.eye(n))
    tau = p.fns[2].params()[0]
    assert 0.5 <= tau <= 2.0 and p.fns[2].kind == wp.FN_EXP_DELAY
    # A1: Bernoulli(0.05) off the diagonal, values in (-1, 1), diagonal 1 + sum |off-diagonal|
    off = A1 - np.diag(np.diag(A1))
    density = np.count_nonzero(off) / (n * (n - 1))
    assert 0.03 < density < 0.07
    assert np.abs(off).max() < 1.0
    assert np.allclose(np.diag(A1) - np.abs(off).sum(axis=1), 1.0)
    # the circle's ends lie strictly between consecutive distinct Laplacian levels
    lev = wp._laplacian_levels(14)
    lo, hi = p.gamma.real - p.a, p.gamma.real + p.a
    for x in (lo, hi):
        j = np.searchsorted(lev, x)
        assert 0 < j < lev.size and lev[j - 1] < x < lev[j]
    assert p.a == p.b and p.gamma.imag == 0.0
    # the drawn members are reproducible
    assert np.array_equal(p.vals, w.config3_member(idx, s=14).vals)
