"""Pins of the oracle's two accuracy measures against values fixed by construction:

  * backward_error: the normwise backward error of the sample solves (reading C5 of the
    sampling step, Algorithm 2 Step 2), eta = ||u - T x||_2 / (||T||_1 ||x||_2 + ||u||_2);
  * eigen_residuals: the eigenpair residual of Section 7.1, ||T(lam) v|| / ||v||, and its
    scaled form ||T(lam) v|| / (||v|| sum_i |f_i(lam)| ||A_i||_F).

Neither pin evaluates the function's own formula on the same data: the residuals are planted
(integer data, so U - T X is exact), the norms are worked out by hand from the matrices'
structure, and the eigenpairs are exact by construction.  A mistake of the kind the pins target
-- the Frobenius or infinity norm in place of the 1-norm, a dropped ||u|| or ||x|| term, a
residual taken from the wrong column, a missing normalisation of v, a coefficient f_i taken
at the wrong point -- changes the value far beyond the tolerances below."""
import numpy as np
import scipy.sparse as sp

import oracle as o
import workloads as w


def _problem(mats, fns, L=1):
    rowptr, colind, vals = w.problems._union(mats)
    n = mats[0].shape[0]
    return w.problems.Problem(name="pin", n=n, rowptr=rowptr, colind=colind, vals=vals, fns=list(fns),
                              gamma=0j, a=1.0, b=1.0, N=1, L=L, U=np.zeros((n, L), dtype=np.complex128, order="F"))


def test_backward_error_hand_example():
    """T = [[1, 2], [0, 3]], x = e_1, u = (1, 4): r = u - T x = (0, 4), ||r|| = 4, ||x|| = 1,
    ||u|| = sqrt(17), ||T||_1 = |2| + |3| = 5 (||T||_inf = 3, ||T||_F = sqrt(14) differ)."""
    A = sp.csr_matrix(np.array([[1.0, 2.0], [0.0, 3.0]]))
    p = _problem([A], [w.Fn(w.FN_CONST)])
    X = np.array([[1.0], [0.0]], dtype=np.complex128)
    U = np.array([[1.0], [4.0]], dtype=np.complex128)
    eta = o.backward_error(p, np.array([1.0 + 0j]), X, U)
    assert eta.shape == (1,)
    assert abs(eta[0] - 4.0 / (5.0 + np.sqrt(17.0))) <= 1e-15
    # an exact solution has eta = 0
    X0 = np.array([[-5.0 / 3.0], [4.0 / 3.0]], dtype=np.complex128)
    assert o.backward_error(p, np.array([1.0 + 0j]), X0, U)[0] <= 1e-16


def test_backward_error_planted_residuals_per_column():
    """T(z) = 2 A_0 + i A_1 with small Gaussian-integer entries, X integer, U = T X + R with a
    planted integer residual R whose columns differ: every quantity is an exact integer, so eta
    per column is known without forming U - T X in floating point."""
    rng = np.random.default_rng(11)
    n, L = 40, 3
    # A_0: tridiagonal real integers; A_1: one heavy column (column 7) plus a diagonal, so that
    # the 1-norm (max column sum) differs from the infinity and Frobenius norms.
    A0 = sp.diags([rng.integers(-3, 4, n - 1), rng.integers(5, 9, n), rng.integers(-3, 4, n - 1)],
                  [-1, 0, 1], dtype=float).toarray()
    A1 = np.diag(rng.integers(-2, 3, n)).astype(float)
    A1[:, 7] += rng.integers(1, 6, n)
    F = np.array([2.0 + 0j, 1j])                     # f_0 = 2, f_1 = i at the point
    T = 2 * A0 + 1j * A1                              # exact: small integers
    p = _problem([sp.csr_matrix(A0), sp.csr_matrix(A1)], [w.Fn(w.FN_CONST), w.Fn(w.FN_CONST)], L)
    X = (rng.integers(-4, 5, (n, L)) + 1j * rng.integers(-4, 5, (n, L))).astype(np.complex128)
    R = np.zeros((n, L), dtype=np.complex128)
    R[3, 0] = 3 + 4j                                  # ||r_0|| = 5
    R[[0, 9], 1] = [12, 5j]                           # ||r_1|| = 13
    # column 2: an exact solution, r_2 = 0
    U = T @ X + R                                     # exact in FP64 (integers << 2^53)
    colsum = np.abs(T).sum(axis=0)                    # |2 a0 + i a1| of integer entries
    norm1 = colsum.max()
    assert norm1 == colsum[7] and norm1 > np.abs(T).sum(axis=1).max()  # the heavy column wins
    eta = o.backward_error(p, F, np.asfortranarray(X), np.asfortranarray(U))
    rn = np.array([5.0, 13.0, 0.0])
    expect = rn / (norm1 * np.linalg.norm(X, axis=0) + np.linalg.norm(U, axis=0))
    assert np.allclose(eta, expect, rtol=1e-13, atol=1e-18)
    assert eta[2] <= 1e-18


def test_eigen_residuals_exact_and_shifted_pairs():
    """T(z) = Q (D - z I) Q^T with Q orthogonal (one Givens rotation per row pair): (d_k, Q e_k)
    is an exact eigenpair; at lam = d_k + delta, T(lam) Q e_k = -delta Q e_k, so the residual is
    |delta| for any scaling of v.  The scaled form divides by ||Q D Q^T||_F + |lam| ||I||_F =
    ||D||_F + |lam| sqrt(n)."""
    n = 8
    d = np.array([1.0, 2.5, -3.0, 4.0, 0.5, 7.0, -1.5, 6.0])
    c, s = np.cos(0.3), np.sin(0.3)
    Q = np.eye(n)
    for k in range(0, n, 2):
        Q[k:k + 2, k:k + 2] = [[c, -s], [s, c]]
    A0 = Q @ np.diag(d) @ Q.T
    A0[np.abs(A0) < 1e-300] = 0.0
    p = _problem([sp.csr_matrix(A0), -sp.identity(n, format="csr")], [w.Fn(w.FN_CONST), w.Fn(w.FN_Z)])
    ks = [1, 4, 6]
    deltas = [0.0, 1e-3, 2.0 - 1.0j]
    lam = np.array([d[k] + dl for k, dl in zip(ks, deltas)], dtype=np.complex128)
    V = np.stack([(3.0 - 4.0j) * Q[:, k] for k in ks], axis=1)   # ||v|| = 5, not normalised
    raw, scaled = o.eigen_residuals(p, lam, V)
    assert raw[0] <= 1e-14
    assert abs(raw[1] - 1e-3) <= 1e-14
    assert abs(raw[2] - abs(2.0 - 1.0j)) <= 1e-13
    norm_terms = np.linalg.norm(d) + np.abs(lam) * np.sqrt(n)
    assert np.allclose(scaled[1:], raw[1:] / norm_terms[1:], rtol=1e-12)


def test_eigen_residuals_function_evaluated_at_lambda():
    """A nonlinear term: T(z) = diag(a) - z I + exp(-z) diag(b).  For v = e_k the residual is
    |a_k - lam + exp(-lam) b_k| exactly, a value computed here from the scalar equation alone."""
    a = np.array([2.0, 3.0, 5.0])
    b = np.array([0.5, -1.0, 2.0])
    p = _problem([sp.diags(a).tocsr(), -sp.identity(3, format="csr"), sp.diags(b).tocsr()],
                 [w.Fn(w.FN_CONST), w.Fn(w.FN_Z), w.Fn(w.FN_EXP_DELAY, (1.0,))])
    lam = np.array([1.0 + 0.5j, 2.0 - 1.0j])
    V = np.eye(3, dtype=np.complex128)[:, [0, 2]]
    raw, scaled = o.eigen_residuals(p, lam, V)
    expect = np.abs(a[[0, 2]] - lam + np.exp(-lam) * b[[0, 2]])
    assert np.allclose(raw, expect, rtol=1e-14)
    norm_terms = np.linalg.norm(a) + np.abs(lam) * np.sqrt(3) + np.abs(np.exp(-lam)) * np.linalg.norm(b)
    assert np.allclose(scaled, expect / norm_terms, rtol=1e-13)
