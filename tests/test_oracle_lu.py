"""Pins for the oracle's FP64 band / dense LU (Algorithm 2, Step 2 solves).

The band LU is checked against LAPACK (numpy / scipy dense routines, which use the same
cabs1 partial-pivoting rule) and against the backward error it must reach in FP64.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle as o


def rand_band(n, kl, ku, rng):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    i, j = np.indices((n, n))
    A[(j - i > ku) | (i - j > kl)] = 0.0
    return A


def to_band(A, kl, ku):
    n = A.shape[0]
    ab = np.zeros((2 * kl + ku + 1, n), dtype=np.complex128, order="F")
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[kl + ku + i - j, j] = A[i, j]
    return ab


SHAPES = [(1, 0, 0), (5, 1, 1), (7, 2, 3), (40, 5, 1), (60, 0, 4), (60, 4, 0), (33, 7, 7), (64, 13, 9)]


@pytest.mark.parametrize("n,kl,ku", SHAPES)
def test_band_lu_matches_lapack_solve(n, kl, ku):
    rng = np.random.default_rng([n, kl, ku])
    A = rand_band(n, kl, ku, rng)
    B = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    ab, ipiv, info = o.band_lu(to_band(A, kl, ku), kl, ku)
    assert info == 0
    X = o.band_solve(ab, ipiv, kl, ku, B)
    Xref = np.linalg.solve(A, B)
    # forward error of two backward-stable solvers: a small multiple of cond(A) u
    bound = 64 * np.linalg.cond(A, 1) * 2.2e-16
    assert np.linalg.norm(X - Xref, 1) <= bound * np.linalg.norm(Xref, 1)
    eta = np.linalg.norm(B - A @ X, axis=0) / (np.abs(A).sum(0).max() * np.linalg.norm(X, axis=0)
                                                + np.linalg.norm(B, axis=0))
    assert eta.max() < 1e-14


@pytest.mark.parametrize("n,kl,ku", SHAPES)
def test_band_pivots_match_lapack_getrf(n, kl, ku):
    # LAPACK zgetrf picks the first entry of largest |re|+|im|; on a banded matrix the
    # band LU must make the same choices (random data: no near-ties).
    rng = np.random.default_rng([n, kl, ku, 1])
    A = rand_band(n, kl, ku, rng)
    _, ipiv, _ = o.band_lu(to_band(A, kl, ku), kl, ku)
    _, piv = sl.lu_factor(A)
    assert np.array_equal(ipiv, piv)


def test_pivot_ties_take_lowest_row():
    # every candidate in column 0 has cabs1 = 2 -> row 0 stays; column 1 then has a unique max
    A = np.array([[1 + 1j, 1, 0], [2, 3, 1], [-1 - 1j, 0, 2]], dtype=np.complex128)
    ab, ipiv, info = o.band_lu(to_band(A, 2, 2), 2, 2)
    assert info == 0
    _, piv = sl.lu_factor(A)
    assert ipiv[0] == 0 == piv[0]
    assert np.array_equal(ipiv, piv)


def test_zero_pivot_reports_first_singular_column():
    A = np.diag([1.0, 2.0, 0.0, 4.0]).astype(np.complex128)
    _, _, info = o.band_lu(to_band(A, 1, 1), 1, 1)
    assert info == 3


def test_dense_lu_matches_lapack():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    B = rng.standard_normal((30, 2)) + 0j
    a, ipiv, info = o.dense_lu(A)
    X = o.dense_solve(a, ipiv, B)
    assert info == 0
    assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-10, atol=1e-12)
    _, piv = sl.lu_factor(A)
    assert np.array_equal(ipiv, piv)


def test_assembly_matches_term_sum():
    import workloads as w
    p = w.config0(N=4, L=2, nx=6, ny=5)
    z = np.array([180.0 + 20j])
    F, _ = o.coefficients(p.fns, z)
    T = o.assemble_dense(p, F[0])
    ref = sum(F[0, i] * p.term(i).toarray() for i in range(p.J))
    assert np.allclose(T, ref, rtol=0, atol=1e-12)
    kl, ku = o.rsrr_oracle.bandwidths(p)
    assert (kl, ku) == (5, 5)
    ab = o.assemble_band(p, F[0], kl, ku)
    assert np.allclose(ab, to_band(ref, kl, ku))
