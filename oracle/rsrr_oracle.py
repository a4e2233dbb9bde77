"""Plain FP64 restatement of RSRR (Algorithm 2) and the modified block SS solver
(Algorithm 1) of Xiao, Meng, Zhang, Zheng (arXiv:1510.07522).

TEST INFRASTRUCTURE: only tests/, the graft smoke check and bench.py's CPU
baseline use this module.  Steps follow the paper's order and notation; the
library primitives used as steps are numpy's SVD/eig/solve and scipy's sparse
products.  Parity pins live in tests/test_oracle_*.py.

Readings of the paper where it is silent or garbled:
  * theta_j = 2 pi (j + 1/2) / N_S for j = 0..N_S-1 (Eq. eq-Ap-num prints j = 0..N_S).
  * V_0 / W_0 are the first nbar columns of V / W (Section 4.3 prints rows).
  * the singular-value gap rule runs over the whole SVD of H (length K k_S).
  * i sqrt(z - s) with branch flag 1 is the continued branch -sqrt(s - z).
  * the sample solves are accepted at normwise backward error
    eta = ||u - T x||_2 / (||T||_1 ||x||_2 + ||u||_2).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.sparse as sp

from . import build as _build

_lib = None


def _clib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        _lib.orc_zgbtrf.argtypes = [i64, i64, i64, p, i64, p]
        _lib.orc_zgbtrf.restype = i64
        _lib.orc_zgbtrs.argtypes = [i64, i64, i64, i64, p, i64, p, p, i64]
        _lib.orc_zgbtrs.restype = None
        _lib.orc_zgetrf.argtypes = [i64, p, i64, p]
        _lib.orc_zgetrf.restype = i64
        _lib.orc_zgetrs.argtypes = [i64, i64, p, i64, p, p, i64]
        _lib.orc_zgetrs.restype = None
    return _lib


# ----------------------------------------------------------------------------------------
# Scalar functions of T(z) = sum_i f_i(z) A_i (Eq. eq-Z-expr) and their derivatives
# (needed by the winding-number count, Eq. eq-ncs).
# ----------------------------------------------------------------------------------------
def coefficients(fns, z):
    """Return (F, dF): arrays [len(z), J] of f_i(z) and f_i'(z)."""
    z = np.asarray(z, dtype=np.complex128)
    F = np.empty(z.shape + (len(fns),), dtype=np.complex128)
    dF = np.empty_like(F)
    for i, fn in enumerate(fns):
        k, p = fn.kind, fn.params()
        if k == 0:
            F[..., i], dF[..., i] = 1.0, 0.0
        elif k == 1:
            F[..., i], dF[..., i] = z, 1.0
        elif k == 2:
            F[..., i], dF[..., i] = z * z, 2.0 * z
        elif k == 3:
            s, branch = p[0], p[1]
            if branch == 0.0:          # i sqrt(z - s), principal root
                r = np.sqrt(z - s)
                F[..., i], dF[..., i] = 1j * r, 0.5j / r
            else:                      # continued branch: i sqrt(z - s) := -sqrt(s - z)
                r = np.sqrt(s - z)
                F[..., i], dF[..., i] = -r, 0.5 / r
        elif k == 4:
            e = np.exp(-p[0] * z)
            F[..., i], dF[..., i] = e, -p[0] * e
        elif k == 5:
            F[..., i] = p[0] * z / (z + p[1])
            dF[..., i] = p[0] * p[1] / (z + p[1]) ** 2
        elif k == 7:                   # Chebyshev polynomial tau_m on [p1, p2] (numpy's chebval)
            m, lo, hi = int(p[0]), p[1], p[2]
            e = np.zeros(m + 1)
            e[m] = 1.0
            x = (2.0 * z - (lo + hi)) / (hi - lo)
            F[..., i] = np.polynomial.chebyshev.chebval(x, e)
            dF[..., i] = np.polynomial.chebyshev.chebval(x, np.polynomial.chebyshev.chebder(e)) * 2.0 / (hi - lo)
        else:
            raise ValueError(f"unknown function kind {k}")
    return F, dF


def contour_points(gamma, a, b, N):
    """Ellipse phi(t) = gamma + a cos t + i b sin t (Eq. eq-contour) at the trapezoid
    nodes theta_j = 2 pi (j + 1/2)/N (Eq. eq-Ap-num); returns (z, dphi, theta)."""
    theta = 2.0 * np.pi * (np.arange(N) + 0.5) / N
    z = gamma + a * np.cos(theta) + 1j * b * np.sin(theta)
    dphi = -a * np.sin(theta) + 1j * b * np.cos(theta)
    return z, dphi, theta


def rectangle_split(N, a, b, side_nodes=0):
    """Points per horizontal and per vertical side of a rectangle with N (even) points."""
    half = N // 2
    nh = side_nodes if side_nodes else int(np.floor(half * a / (a + b) + 0.5))
    nh = min(max(nh, 1), half - 1)
    return nh, half - nh


def contour_rule(gamma, a, b, N, shape="ellipse", side_nodes=0):
    """Nodes z_j and weights w_j with (1 / 2 pi i) oint g(z) dz ~ sum_j w_j g(z_j).

    ellipse:   the trapezoid rule of Eq. eq-Ap-num, w_j = phi'(theta_j) / (i N).
    rectangle: gamma + [-a, a] + i [-b, b] counter-clockwise from the lower-left corner
               (bottom, right, top, left), an m-point Gauss-Legendre rule on each side
               (Section 7.2, the gun example); on a side from P to Q, z = P + (Q - P)(t + 1)/2
               and dz = (Q - P)/2 dt.
    """
    if shape == "ellipse":
        z, dphi, _ = contour_points(gamma, a, b, N)
        return z, dphi / (1j * N)
    assert shape == "rectangle" and N % 2 == 0 and N >= 4
    nh, nv = rectangle_split(N, a, b, side_nodes)
    corners = [gamma - a - 1j * b, gamma + a - 1j * b, gamma + a + 1j * b, gamma - a + 1j * b]
    zs, ws = [], []
    for side in range(4):
        P, Q = corners[side], corners[(side + 1) % 4]
        t, om = np.polynomial.legendre.leggauss(nh if side % 2 == 0 else nv)
        zs.append(P + (Q - P) * (t + 1) / 2)
        ws.append(om * (Q - P) / 2 / (2j * np.pi))
    return np.concatenate(zs), np.concatenate(ws)


def inside_contour(lam, gamma, a, b, shape="ellipse"):
    w = np.asarray(lam) - gamma
    if shape == "rectangle":
        return (np.abs(w.real) < a) & (np.abs(w.imag) < b)
    return (w.real / a) ** 2 + (w.imag / b) ** 2 < 1.0


def _is_tz(prob):
    return getattr(prob, "tz", None) is not None


def _T_at(prob, z):
    """T(z) as a sparse matrix on the pattern (from the values of a tz problem, or sum f_i A_i)."""
    if _is_tz(prob):
        v = prob.tz(z)
    else:
        F, _ = coefficients(prob.fns, np.array([z]))
        v = F[0] @ prob.vals
    return sp.csr_matrix((v, prob.colind, prob.rowptr), shape=(prob.n, prob.n))


def _shape(prob):
    return getattr(prob, "shape", "ellipse"), getattr(prob, "side_nodes", 0)


# ----------------------------------------------------------------------------------------
# Assembly of T(z) (Eq. eq-Z-expr) and the band solves of Algorithm 2, Step 2.
# ----------------------------------------------------------------------------------------
def _rows(prob):
    return np.repeat(np.arange(prob.n, dtype=np.int64), np.diff(prob.rowptr))


def assemble_values(prob, Frow):
    """Values of T(z) on the union pattern: sum_i f_i(z) A_i."""
    return Frow @ prob.vals


def assemble_dense(prob, Frow):
    T = np.zeros((prob.n, prob.n), dtype=np.complex128)
    np.add.at(T, (_rows(prob), prob.colind), assemble_values(prob, Frow))
    return T


def bandwidths(prob):
    d = prob.colind.astype(np.int64) - _rows(prob)
    return int(max(0, -d.min())), int(max(0, d.max()))


def assemble_band(prob, Frow, kl, ku):
    """T(z) in general-band layout (ldab = 2 kl + ku + 1, fill rows zero)."""
    ldab = 2 * kl + ku + 1
    ab = np.zeros((ldab, prob.n), dtype=np.complex128, order="F")
    r, c = _rows(prob), prob.colind.astype(np.int64)
    np.add.at(ab, (kl + ku + r - c, c), assemble_values(prob, Frow))
    return ab


def band_lu(ab, kl, ku):
    ab = np.asfortranarray(ab, dtype=np.complex128).copy(order="F")
    n = ab.shape[1]
    ipiv = np.zeros(n, dtype=np.int32)
    info = _clib().orc_zgbtrf(n, kl, ku, ab.ctypes.data, ab.shape[0], ipiv.ctypes.data)
    return ab, ipiv, int(info)


def band_solve(ab, ipiv, kl, ku, B):
    X = np.asfortranarray(B, dtype=np.complex128).copy(order="F")
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n = ab.shape[1]
    _clib().orc_zgbtrs(n, kl, ku, X.shape[1], ab.ctypes.data, ab.shape[0], ipiv.ctypes.data,
                       X.ctypes.data, X.shape[0])
    return X


def dense_lu(A):
    a = np.asfortranarray(A, dtype=np.complex128).copy(order="F")
    ipiv = np.zeros(a.shape[0], dtype=np.int32)
    info = _clib().orc_zgetrf(a.shape[0], a.ctypes.data, a.shape[0], ipiv.ctypes.data)
    return a, ipiv, int(info)


def dense_solve(a, ipiv, B):
    X = np.asfortranarray(B, dtype=np.complex128).copy(order="F")
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    _clib().orc_zgetrs(a.shape[0], X.shape[1], a.ctypes.data, a.shape[0], ipiv.ctypes.data,
                       X.ctypes.data, X.shape[0])
    return X


def one_norm(prob, Frow):
    """||T(z)||_1 = max column sum of |T_ij|."""
    col = np.zeros(prob.n)
    np.add.at(col, prob.colind, np.abs(assemble_values(prob, Frow)))
    return float(col.max())


def backward_error(prob, Frow, X, U):
    """Columnwise eta = ||u - T x|| / (||T||_1 ||x|| + ||u||) (normwise, Rigal-Gaches)."""
    T = sp.csr_matrix((assemble_values(prob, Frow), prob.colind, prob.rowptr), shape=(prob.n, prob.n))
    R = U - T @ X
    return np.linalg.norm(R, axis=0) / (one_norm(prob, Frow) * np.linalg.norm(X, axis=0)
                                        + np.linalg.norm(U, axis=0))


def _solve_point(prob, Frow, kl, ku, dense):
    if dense:
        a, ipiv, info = dense_lu(assemble_dense(prob, Frow))
        X = dense_solve(a, ipiv, prob.U)
    else:
        ab, ipiv, info = band_lu(assemble_band(prob, Frow, kl, ku), kl, ku)
        X = band_solve(ab, ipiv, kl, ku, prob.U)
    return X, info


def sample(prob, points=None, threads=None, dense=False, z=None):
    """Algorithm 2, Step 2 and Eq. eq-hatS: S_hat = [T(z_0)^{-1} U, ..., T(z_{N-1})^{-1} U].

    `points` restricts the work to a subset of the sampling indices (returns only those
    column blocks).  Returns (S_hat [n, len(points) L], info per point, eta per column).
    """
    if z is None:
        shape, side_nodes = _shape(prob)
        z, _ = contour_rule(prob.gamma, prob.a, prob.b, prob.N, shape, side_nodes)
    pts = list(range(len(z))) if points is None else list(points)
    if _is_tz(prob):
        # T known by its values: T(z_j) of each sampling point as its own term, coefficients I
        prob = dataclasses.replace(prob, vals=np.stack([prob.tz(zz) for zz in z]), fns=[])
        F = np.eye(len(z), dtype=np.complex128)
    else:
        F, _ = coefficients(prob.fns, z)
    kl, ku = bandwidths(prob)
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(lambda j: _solve_point(prob, F[j], kl, ku, dense), pts))
    Shat = np.empty((prob.n, len(pts) * prob.L), dtype=np.complex128, order="F")
    infos, etas = [], []
    for k, (j, (X, info)) in enumerate(zip(pts, res)):
        Shat[:, k * prob.L:(k + 1) * prob.L] = X
        infos.append(info)
        etas.append(backward_error(prob, F[j], X, prob.U))
    return Shat, np.array(infos), np.concatenate(etas) if etas else np.zeros(0)


# ----------------------------------------------------------------------------------------
# Algorithm 2, Step 3: truncated SVD of S_hat (keep sigma_k > delta sigma_1).
# ----------------------------------------------------------------------------------------
def numerical_rank(sigma, delta):
    sigma = np.asarray(sigma)
    if sigma.size == 0 or sigma[0] == 0.0:
        return 0
    return int(np.count_nonzero(sigma > delta * sigma[0]))


def truncated_basis(Shat, delta=1e-14):
    Ub, sigma, _ = np.linalg.svd(Shat, full_matrices=False)
    k = numerical_rank(sigma, delta)
    return np.asfortranarray(Ub[:, :k]), sigma, k


# ----------------------------------------------------------------------------------------
# The moment scheme of SSRR (Section 3.1, Eqs. eq-malpha-qud and eq-hatM): the projection space
# is spanned by the quadrature moments M_alpha = sum_i w_i z_i^alpha T(z_i)^{-1} U, alpha < K',
# instead of by the samples themselves.  w_i = phi'(theta_i) / (i N) are the trapezoid weights
# of (1 / 2 pi i) oint dz on the ellipse.  The monomials are taken in the shifted and scaled
# variable (z - gamma) / rho with rho = max(a, b): a polynomial change of basis of degree < K',
# so span(M_hat) is the same, with better-scaled columns.
# ----------------------------------------------------------------------------------------
def moment_matrix(prob, Shat, Kp):
    shape, side_nodes = _shape(prob)
    z, w = contour_rule(prob.gamma, prob.a, prob.b, prob.N, shape, side_nodes)
    rho = max(prob.a, prob.b)
    zeta = (z - prob.gamma) / rho
    L = prob.L
    M = np.zeros((prob.n, Kp * L), dtype=np.complex128, order="F")
    for al in range(Kp):
        for i in range(prob.N):
            M[:, al * L:(al + 1) * L] += w[i] * zeta[i] ** al * Shat[:, i * L:(i + 1) * L]
    return M


# ----------------------------------------------------------------------------------------
# Section 6.2 (Eqs. eq-T-interp, eq-T-coefs, eq-Ts-interp, eq-Ts-coefs): the reduced NEP as a
# Chebyshev interpolant of degree d on the real interval [lo, hi].  The paper states the rule
# on [-1, 1]; x = c + r t maps it (c, r the centre and half-width).  Its coefficient formula
# read literally doubles the constant term; the first-kind interpolant takes half of it for
# j = 0 (the reading that reproduces polynomials of degree <= d exactly).
# ----------------------------------------------------------------------------------------
def chebyshev_reduce(prob, S, d, lo, hi):
    """Returns (P_hat [d+1, k, k], fns): T_S(z) ~ sum_j P_hat_j tau_j((2z - lo - hi)/(hi - lo))."""
    m = d + 1
    c, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
    theta = (np.arange(m) + 0.5) * np.pi / m
    x = c + r * np.cos(theta)
    Q = []
    for k in range(m):
        Tk = _T_at(prob, x[k])
        Q.append(S.conj().T @ (Tk @ S))
    Phat = np.zeros((m,) + Q[0].shape, dtype=np.complex128)
    for j in range(m):
        for k in range(m):
            Phat[j] += (2.0 / m) * np.cos(j * theta[k]) * Q[k]
    Phat[0] *= 0.5
    fns = [_Fn(7, (float(j), float(lo), float(hi))) for j in range(m)]
    return Phat, fns


class _Fn:
    """A function descriptor of the reduced NEP (kind and parameters, as in the workloads)."""
    def __init__(self, kind, p):
        self.kind, self.p = kind, tuple(p)

    def params(self):
        q = list(self.p) + [0.0] * 4
        return [float(v) for v in q[:4]]


# ----------------------------------------------------------------------------------------
# Algorithm 2, Step 4 (first half), Eq. eq-Zs-expr: P_i = S^H A_i S.
# ----------------------------------------------------------------------------------------
def project(prob, S):
    return np.stack([S.conj().T @ (prob.term(i) @ S) for i in range(prob.J)])


# ----------------------------------------------------------------------------------------
# Algorithm 1: modified block SS for T_S(z) = sum_i f_i(z) P_i.
# ----------------------------------------------------------------------------------------
def _reduced_T(P, Frow):
    return np.tensordot(Frow, P, axes=(0, 0))


def reduced_ss(P, fns, gamma, a, b, N_S=500, K=2, tol_gap=1e3, return_diag=False, shape="ellipse"):
    """Returns (lam [nbar], g [k_S, nbar]) plus diagnostics if requested.

    Step 2: moments A_alpha (Eq. eq-Ap-num, rho = max(a, b); on a rectangle the Gauss-Legendre
            rule of contour_rule with N_S points split in proportion to the sides) and
            H, H^< (Eq. eq-HH).
    Step 3: SVD of H (Eq. eq-svdH) and nbar from the winding number (Eq. eq-ncs) and the
            singular-value gap (Eq. eq-gap), combined as Section 4.3 suggests.
    Step 4: A = V_0^H H^< W_0 Sigma_0^{-1} (Eq. eq-A), eig, then Eq. eq-eigens.
    """
    k = P.shape[1]
    rho = max(a, b)
    z, wq = contour_rule(gamma, a, b, N_S, shape)
    F, dF = coefficients(fns, z)
    moments = np.zeros((2 * K, k, k), dtype=np.complex128)
    wind = 0.0 + 0.0j
    for j in range(N_S):
        Ts = _reduced_T(P, F[j])
        Tinv = np.linalg.solve(Ts, np.eye(k))
        dTs = _reduced_T(P, dF[j])
        wind += np.trace(Tinv @ dTs) * wq[j]
        w = (z[j] - gamma) / rho
        for al in range(2 * K):
            moments[al] += (w ** al) * wq[j] * Tinv
    H = np.block([[moments[r + c] for c in range(K)] for r in range(K)])
    Hl = np.block([[moments[r + c + 1] for c in range(K)] for r in range(K)])
    V, sig, Wh = np.linalg.svd(H)
    W = Wh.conj().T
    n_w = int(np.rint(wind.real))
    gaps = sig[:-1] / np.maximum(sig[1:], 1e-300)
    n_g = int(np.argmax(gaps)) + 1 if gaps.size and gaps.max() >= tol_gap else None

    def extract(nb):
        if nb <= 0:
            return np.zeros(0, np.complex128), np.zeros((k, 0), np.complex128)
        V0, S0, W0 = V[:, :nb], sig[:nb], W[:, :nb]
        A = V0.conj().T @ Hl @ W0 / S0[None, :]
        lp, gp = np.linalg.eig(A)
        Hr = np.hstack([moments[al] for al in range(K)])
        g = Hr @ (W0 / S0[None, :]) @ gp
        return rho * lp + gamma, g

    def max_red_res(lam, g):
        if lam.size == 0:
            return 0.0
        Fl, _ = coefficients(fns, lam)
        r = [np.linalg.norm(_reduced_T(P, Fl[t]) @ g[:, t]) / np.linalg.norm(g[:, t])
             for t in range(lam.size)]
        return float(max(r))

    if n_w <= 0:
        nbar = 0
    elif n_g is None or n_g == n_w:
        nbar = n_w
    else:
        cand = [(max_red_res(*extract(nn)), nn) for nn in (n_w, n_g)]
        nbar = min(cand)[1]
    nbar = min(nbar, K * k)
    lam, g = extract(nbar)
    if return_diag:
        return lam, g, dict(winding=wind, n_winding=n_w, n_gap=n_g, sigma_H=sig, nbar=nbar,
                            moments=moments)
    return lam, g


# ----------------------------------------------------------------------------------------
# Algorithm 2, Step 5 and the residual of Section 7.1.
# ----------------------------------------------------------------------------------------
def backmap(S, g):
    V = S @ g
    return V / np.linalg.norm(V, axis=0, keepdims=True)


def eigen_residuals(prob, lam, V):
    """(raw ||T(lam) v|| / ||v||, scaled raw / sum_i |f_i(lam)| ||A_i||_F) per pair; for a tz
    problem (no A_i) the scale is ||T(lam)||_F."""
    raw, scaled = [], []
    for t in range(len(lam)):
        T = _T_at(prob, lam[t])
        r = np.linalg.norm(T @ V[:, t]) / np.linalg.norm(V[:, t])
        raw.append(r)
        if _is_tz(prob):
            scaled.append(r / np.linalg.norm(T.data))
        else:
            F, _ = coefficients(prob.fns, np.array([lam[t]]))
            normA = np.array([np.linalg.norm(prob.vals[i]) for i in range(prob.J)])
            scaled.append(r / float(np.abs(F[0]) @ normA))
    return np.array(raw), np.array(scaled)


def rsrr(prob, delta=1e-14, N_S=500, K=2, tol_gap=1e3, threads=None, dense=False, moments=0, z=None,
         chebyshev=None):
    """Algorithm 2 end to end; eigenvalues strictly inside the ellipse, sorted by |lam|.
    moments = K' > 0: the SSRR moment scheme (Step 3 on M_hat of K' moments instead of S_hat).
    z: sampling points other than the contour's nodes (Section 3.2 allows any points in the
    domain; the ellipse still bounds Algorithm 1).
    chebyshev = (d, lo, hi): the reduced NEP as its Chebyshev interpolant (Section 6.2)."""
    assert not (moments and z is not None), "the moment scheme needs the contour's nodes"
    Shat, infos, eta = sample(prob, threads=threads, dense=dense, z=z)
    S, sigma, k_S = truncated_basis(moment_matrix(prob, Shat, moments) if moments else Shat, delta)
    if chebyshev is None:
        assert not _is_tz(prob), "a tz problem has no A_i: use the Chebyshev route"
        P, rfns = project(prob, S), prob.fns
    else:
        P, rfns = chebyshev_reduce(prob, S, *chebyshev)
    shape, _ = _shape(prob)
    lam, g, diag = reduced_ss(P, rfns, prob.gamma, prob.a, prob.b, N_S, K, tol_gap,
                              return_diag=True, shape=shape)
    keep = inside_contour(lam, prob.gamma, prob.a, prob.b, shape)
    lam, g = lam[keep], g[:, keep]
    order = np.argsort(np.abs(lam), kind="stable")
    lam, g = lam[order], g[:, order]
    V = backmap(S, g)
    raw, scaled = eigen_residuals(prob, lam, V)
    return dict(lam=lam, V=V, resid=raw, resid_scaled=scaled, k_S=k_S, sigma=sigma, P=P,
                S=S, Shat=Shat, eta=eta, infos=infos, **diag)
