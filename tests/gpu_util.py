"""Helpers shared by the GPU tests: marshal a workloads.Problem through the C ABI."""
import numpy as np
import scipy.sparse as sp

import workloads


def fns_of(prob):
    return [(f.kind, f.params()) for f in prob.fns]


def open_nep(rs, prob, flags=0):
    return rs.Nep(prob.n, prob.rowptr, prob.colind, prob.vals, fns_of(prob), flags)


def scrambled(prob, seed=1):
    """The same NEP with rows and columns permuted at random (destroys the natural band)."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(prob.n)
    mats = []
    for i in range(prob.J):
        A = prob.term(i).tocsr()
        mats.append(A[p][:, p])
    rowptr, colind, vals = workloads.problems._union(mats)
    q = workloads.problems.Problem(name=prob.name + "_scrambled", n=prob.n, rowptr=rowptr, colind=colind,
                                   vals=vals, fns=prob.fns, gamma=prob.gamma, a=prob.a, b=prob.b, N=prob.N,
                                   L=prob.L, U=np.asfortranarray(prob.U[p]), seed=prob.seed, meta=dict(prob.meta))
    return q, p


def rel_err_cols(X, Y):
    return np.linalg.norm(X - Y, axis=0) / np.linalg.norm(Y, axis=0)


def match(a, b):
    from scipy.optimize import linear_sum_assignment
    a, b = np.asarray(a), np.asarray(b)
    assert a.size == b.size, (a.size, b.size)
    if a.size == 0:
        return 0.0
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    return float(np.max(np.abs(a[r] - b[c]) / np.abs(b[c])))
