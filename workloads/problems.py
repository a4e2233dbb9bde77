"""Seeded NEP generators: T(z) = sum_i f_i(z) A_i over one union sparsity pattern.

The affine-in-functions form is the paper's Eq. (eq-Z-expr) (Section 6); every
generator returns the matrices A_i, the function descriptors (kind, params) of
f_i, an elliptic contour phi(t) = gamma + a cos t + i b sin t (Eq. eq-contour),
the sample count N, the probe width L, and a seeded probing matrix U
(Algorithm 2, Step 1).  Nothing here evaluates f_i or touches T(z).

Index convention for grid problems: node (ix, iy) of an nx-by-ny interior grid
has index ix*ny + iy (y fastest), so the natural order is already banded with
semi-bandwidth ny.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

# Function kinds; the integer values are the C ABI's rsrr_fkind values.
FN_CONST = 0        # f = 1
FN_Z = 1            # f = z
FN_Z2 = 2           # f = z^2
FN_ISQRT_SHIFT = 3  # f = i*sqrt(z - p0); p1 = 0 principal branch, p1 = 1 continued branch -sqrt(p0 - z)
FN_EXP_DELAY = 4    # f = exp(-p0 z)
FN_RATIONAL = 5     # f = p0 z / (z + p1)
FN_CHEBYSHEV = 7    # f = tau_{p0}((2z - p1 - p2) / (p2 - p1)), Chebyshev polynomial on [p1, p2]


@dataclass
class Fn:
    kind: int
    p: Sequence[float] = (0.0, 0.0, 0.0, 0.0)

    def params(self):
        q = list(self.p) + [0.0] * 4
        return [float(x) for x in q[:4]]


@dataclass
class Problem:
    """One NEP instance plus its RSRR sampling parameters."""
    name: str
    n: int
    rowptr: np.ndarray          # int64 [n+1], union pattern (rows sorted by column)
    colind: np.ndarray          # int32 [nnz]
    vals: np.ndarray            # complex128 [J, nnz], aligned to the union pattern
    fns: List[Fn]
    gamma: complex              # contour centre
    a: float                    # real semi-axis
    b: float                    # imaginary semi-axis
    N: int                      # sampling points on the contour
    L: int                      # probing columns
    U: np.ndarray               # complex128 [n, L] (Fortran order)
    seed: int = 0
    meta: dict = field(default_factory=dict)
    shape: str = "ellipse"      # or "rectangle": gamma + [-a, a] + i [-b, b]
    side_nodes: int = 0         # rectangle: sampling points per horizontal side (0 = proportional)

    @property
    def J(self) -> int:
        return self.vals.shape[0]

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def term(self, i: int) -> sp.csr_matrix:
        """A_i as a scipy CSR matrix on the union pattern (explicit zeros kept)."""
        return sp.csr_matrix((self.vals[i], self.colind, self.rowptr), shape=(self.n, self.n))

    def vals_reim(self) -> np.ndarray:
        """float64 [J, nnz, 2] view (interleaved re/im), the ABI's value layout."""
        return np.ascontiguousarray(self.vals).view(np.float64).reshape(self.J, self.nnz, 2)


@dataclass
class TzProblem(Problem):
    """A NEP known only by its values: tz(z) -> complex [nnz], T(z) on the pattern.  vals is
    empty (J = 0) and fns too; tz is the problem's definition, as a BEM assembly routine would
    be, not a step of the method."""
    tz: Optional[object] = None


def probe_matrix(n: int, L: int, seed: int) -> np.ndarray:
    """Random complex Gaussian U (n x L): re, im iid N(0,1)/sqrt(2) (Algorithm 2, Step 1)."""
    g = np.random.default_rng(seed).standard_normal((L, n, 2))
    U = (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)
    return np.asfortranarray(U.T)


def grid_laplacian(nx: int, ny: int, hx: float, hy: float) -> sp.csr_matrix:
    """5-point Dirichlet Laplacian, -d2/dx2 - d2/dy2, index ix*ny + iy."""
    ex = np.ones(nx)
    ey = np.ones(ny)
    Dx = sp.diags([-ex[1:], 2 * ex, -ex[1:]], [-1, 0, 1], shape=(nx, nx), dtype=np.float64) / hx ** 2
    Dy = sp.diags([-ey[1:], 2 * ey, -ey[1:]], [-1, 0, 1], shape=(ny, ny), dtype=np.float64) / hy ** 2
    return (sp.kron(Dx, sp.identity(ny)) + sp.kron(sp.identity(nx), Dy)).tocsr()


def _union(mats: Sequence[sp.spmatrix]):
    """Align several sparse matrices to their union pattern (sorted CSR)."""
    n = mats[0].shape[0]
    pat = None
    for m in mats:
        c = sp.coo_matrix(m)
        q = sp.csr_matrix((np.ones(c.nnz), (c.row, c.col)), shape=(n, n))
        pat = q if pat is None else (pat + q)
    pat = pat.tocsr()
    pat.sort_indices()
    pat.data[:] = 1.0
    rowptr = pat.indptr.astype(np.int64)
    colind = pat.indices.astype(np.int32)
    vals = np.zeros((len(mats), pat.nnz), dtype=np.complex128)
    # position of (r, c) in the union pattern via a key search
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    keys = rows * n + colind.astype(np.int64)
    for i, m in enumerate(mats):
        c = sp.coo_matrix(m)
        k = c.row.astype(np.int64) * n + c.col.astype(np.int64)
        pos = np.searchsorted(keys, k)
        np.add.at(vals[i], pos, c.data.astype(np.complex128))
    return rowptr, colind, vals


def _make(name, mats, fns, gamma, a, b, N, L, seed, meta):
    rowptr, colind, vals = _union(mats)
    n = mats[0].shape[0]
    return Problem(name=name, n=n, rowptr=rowptr, colind=colind, vals=vals, fns=list(fns),
                   gamma=complex(gamma), a=float(a), b=float(b), N=int(N), L=int(L),
                   U=probe_matrix(n, L, seed), seed=seed, meta=meta)


# --------------------------------------------------------------------------------------
# Gun-like square-root NEP: T(z) = K - z M + i sqrt(z - s1) W1 + i sqrt(z - s2) W2.
# W1 / W2 are 0/1 masks of the nodes with ix = 0 / ix = nx-1.  The s2 term uses the
# continued branch i*sqrt(z - s2) := -sqrt(s2 - z) so it is holomorphic inside the
# contour (the principal cut of sqrt(z - s2) would cross it on the real axis).
# --------------------------------------------------------------------------------------
def _gun_like(name, nx, ny, hx, hy, gamma, radius, N, L, seed=0, sigma1=0.0, sigma2=108.8,
              with_masks=True):
    K = grid_laplacian(nx, ny, hx, hy)
    n = nx * ny
    M = sp.identity(n, format="csr")
    w1 = np.zeros(n)
    w1[:ny] = 1.0
    w2 = np.zeros(n)
    w2[(nx - 1) * ny:] = 1.0
    mats = [K, -M]
    fns = [Fn(FN_CONST), Fn(FN_Z)]
    if with_masks:
        mats += [sp.diags(w1).tocsr(), sp.diags(w2).tocsr()]
        fns += [Fn(FN_ISQRT_SHIFT, (sigma1 ** 2, 0.0)), Fn(FN_ISQRT_SHIFT, (sigma2 ** 2, 1.0))]
    meta = dict(nx=nx, ny=ny, hx=hx, hy=hy, band=ny, sigma1=sigma1, sigma2=sigma2)
    return _make(name, mats, fns, gamma, radius, radius, N, L, seed, meta)


def config0(N=32, L=16, nx=30, ny=30):
    """30x30 gun-like sqrt NEP, circle (250, 150), N=32, L=16, complex128."""
    return _gun_like("config0", nx, ny, 1.0 / (nx + 1), 1.0 / (ny + 1), 250.0, 150.0, N, L)


def config0_linear(N=32, L=16, nx=30, ny=30):
    """config0 without the masks: T(z) = K - z I, eigenvalues in closed form."""
    return _gun_like("config0_linear", nx, ny, 1.0 / (nx + 1), 1.0 / (ny + 1), 250.0, 150.0,
                     N, L, with_masks=False)


def config0_rect(N=30, L=4, side_nodes=10, linear=False):
    """config0's NEP (or its linear part) with the paper's gun-example contour shape: a
    rectangle of 195.4 x 50 (lower-left 140 - 5i, upper-right 335.4 + 45i; shifted 5 below
    the real axis, which the eigenvalues here lie just above) with N Gauss-Legendre points,
    side_nodes on each long side ("10-5" for N = 30)."""
    p = config0_linear(N=N, L=L) if linear else config0(N=N, L=L)
    p.name = "config0_rect_linear" if linear else "config0_rect"
    p.gamma, p.a, p.b = complex(237.7, 20.0), 97.7, 25.0
    p.shape, p.side_nodes = "rectangle", int(side_nodes)
    return p


def config2(N=64, L=48, nx=400, ny=250, gamma=330.0, radius=300.0):
    """400x250 gun-like sqrt NEP (band 250), circle centre 330, radius 300, N=64, L=48."""
    return _gun_like("config2", nx, ny, 1.0 / (nx + 1), 1.0 / (ny + 1), gamma, radius, N, L)


# --------------------------------------------------------------------------------------
# Damped quadratic NEP T(z) = K + z C + z^2 M, C = 0.05 K + 0.02 M (Rayleigh damping).
# --------------------------------------------------------------------------------------
def _damped_mats(s):
    h = 1.0 / (s + 1)
    K = grid_laplacian(s, s, h, h)
    n = s * s
    rng = np.random.default_rng([1, 0])
    m = 1.0 + 0.1 * rng.random(n)
    M = sp.diags(m).tocsr()
    C = (0.05 * K + 0.02 * M).tocsr()
    return K, C, M, m


def config1(s=200, N=64, L=32):
    """200x200 damped QEP (band 200), ellipse centre -0.5+40i, semi-axes 2 (re) x 30 (im)."""
    K, C, M, _ = _damped_mats(s)
    return _make("config1", [K, C, M], [Fn(FN_CONST), Fn(FN_Z), Fn(FN_Z2)],
                 -0.5 + 40j, 2.0, 30.0, N, L, 0, dict(nx=s, ny=s, band=s, alpha=0.05, beta=0.02))


def damped_eigs(s, count):
    """Upper-branch eigenvalues z of K + z C + z^2 M for the `count` smallest mu of K v = mu M v.

    Used only to place the config-1b contour (input preparation): with C = a K + b M,
    T(z) v = 0 iff z^2 + (b + a mu) z + mu = 0.
    """
    K, _, _, m = _damped_mats(s)
    n = s * s
    if n <= 4000:
        Mi = 1.0 / np.sqrt(m)
        A = (sp.diags(Mi) @ K @ sp.diags(Mi)).toarray()
        mu = np.linalg.eigvalsh(A)[:count]
    else:
        import scipy.sparse.linalg as sla
        mu = np.sort(sla.eigsh(K.tocsc(), k=count, M=sp.diags(m).tocsc(), sigma=0.0,
                               which="LM", return_eigenvectors=False))
    c = 0.02 + 0.05 * mu
    return (-c + 1j * np.sqrt(4 * mu - c * c + 0j)) / 2.0


def config1b(s=200, N=64, L=32, m=10):
    """config1's matrices with an ellipse placed around the m lowest upper-branch eigenvalues.

    The ellipse's real extent is set by the real parts of those eigenvalues, its imaginary
    extent by the gap midpoints to the next eigenvalue on either side.  Near the ends of the
    real range the ellipse narrows, so the outermost of the m can fall outside it (s = 200:
    8 of 10 inside); users count the enclosed ones with the contour test.
    """
    K, C, M, _ = _damped_mats(s)
    z = damped_eigs(s, m + 1)
    inside, nxt = z[:m], z[m]
    lo_im = 0.5 * inside.imag.min()              # midpoint between conjugate branches
    hi_im = 0.5 * (inside.imag.max() + nxt.imag) if nxt.imag > inside.imag.max() else inside.imag.max() * 1.05
    re_lo = inside.real.min() - 0.5
    re_hi = inside.real.max() + 0.5
    gamma = complex(0.5 * (re_lo + re_hi), 0.5 * (lo_im + hi_im))
    a = 0.5 * (re_hi - re_lo) * 1.6
    b = 0.5 * (hi_im - lo_im)
    return _make("config1b", [K, C, M], [Fn(FN_CONST), Fn(FN_Z), Fn(FN_Z2)],
                 gamma, a, b, N, L, 0, dict(nx=s, ny=s, band=s, expected=z[:m]))


# --------------------------------------------------------------------------------------
# Time-delay NEP T(z) = -z I + A0 + A1 exp(-tau z) (batch member).
# --------------------------------------------------------------------------------------
def _laplacian_levels(s):
    """Distinct eigenvalues of the s x s unit-square Dirichlet Laplacian (h = 1/(s+1))."""
    h = 1.0 / (s + 1)
    k = np.arange(1, s + 1)
    lam1 = 4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
    lev = np.unique(np.round((lam1[:, None] + lam1[None, :]).ravel(), 9))
    return lev


def config3_member(idx, s=None, N=32, L=8, master_seed=3, tau=None):
    """Member `idx` of the time-delay batch; A0 = (s+1)^2 * 5-point, A1 Bernoulli(0.05).
    `tau` overrides the drawn delay (tau = 0 makes T linear: -zI + A0 + A1)."""
    rng = np.random.default_rng([master_seed, 0, idx])
    if s is None:
        s = int(rng.integers(20, 101))
    tau_drawn = float(rng.uniform(0.5, 2.0))
    tau = tau_drawn if tau is None else float(tau)
    n = s * s
    h = 1.0 / (s + 1)
    A0 = grid_laplacian(s, s, h, h)
    mask = rng.random((n, n)) < 0.05 if n <= 3000 else None
    if mask is None:
        nnz_target = int(0.05 * n * n)
        r = rng.integers(0, n, nnz_target)
        c = rng.integers(0, n, nnz_target)
        keep = r != c
        A1 = sp.coo_matrix((rng.uniform(-1, 1, keep.sum()), (r[keep], c[keep])), shape=(n, n)).tocsr()
        A1.sum_duplicates()
    else:
        np.fill_diagonal(mask, False)
        r, c = np.nonzero(mask)
        A1 = sp.coo_matrix((rng.uniform(-1, 1, r.size), (r, c)), shape=(n, n)).tocsr()
    rowsum = np.asarray(abs(A1).sum(axis=1)).ravel()
    A1 = (A1 + sp.diags(1.0 + rowsum)).tocsr()
    lev = _laplacian_levels(s)
    k0 = int(rng.integers(2, 7))
    m = int(rng.integers(4, 13))
    lo = 0.5 * (lev[k0 - 2] + lev[k0 - 1])
    hi = 0.5 * (lev[k0 + m - 1] + lev[k0 + m])
    I = sp.identity(n, format="csr")
    return _make(f"config3[{idx}]", [-I, A0, A1],
                 [Fn(FN_Z), Fn(FN_CONST), Fn(FN_EXP_DELAY, (tau,))],
                 0.5 * (lo + hi), 0.5 * (hi - lo), 0.5 * (hi - lo), N, L, 0,
                 dict(nx=s, ny=s, band=n - 1, tau=tau, k0=k0, m=m))


def config3_batch(count=256, N=32, L=8):
    return [config3_member(i, N=N, L=L) for i in range(count)]


# --------------------------------------------------------------------------------------
# Small pinned problems.
# --------------------------------------------------------------------------------------
def _banded_orthogonal(n, rng, sweeps=2):
    """Q = product of adjacent Givens rotations (band 2*sweeps), returned dense."""
    Q = np.eye(n)
    for s in range(sweeps):
        for i in range(s % 2, n - 1, 2):
            t = rng.uniform(0, 2 * np.pi)
            c, si = np.cos(t), np.sin(t)
            G = np.eye(n)
            G[i, i] = c
            G[i, i + 1] = -si
            G[i + 1, i] = si
            G[i + 1, i + 1] = c
            Q = Q @ G
    return Q


def planted_sqrt(n=24, seed=7, N=48, L=4, sigma=None):
    """T(z) = Q (D0 - z I + i sqrt(z) D1 + i sqrt(z - sigma^2) D2) Q^T with Q banded orthogonal.

    Each diagonal entry is a scalar NEP, so the eigenvalues are those of the scalar
    equations d0 - z + i d1 sqrt(z) (+ ...) = 0.  With sigma=None the D2 term is absent
    and w = sqrt(z) solves w^2 - i d1 w - d0 = 0 exactly.
    """
    rng = np.random.default_rng([11, seed])
    Q = _banded_orthogonal(n, rng)
    d0 = np.sort(rng.uniform(50, 300, n))
    d1 = rng.uniform(0.5, 2.0, n)
    Qs = sp.csr_matrix(np.where(np.abs(Q) > 0, Q, 0))
    def conj(d):
        return sp.csr_matrix(Q @ np.diag(d) @ Q.T)
    mats = [conj(d0), -sp.csr_matrix(np.eye(n)), conj(d1)]
    fns = [Fn(FN_CONST), Fn(FN_Z), Fn(FN_ISQRT_SHIFT, (0.0, 0.0))]
    meta = dict(d0=d0, d1=d1, Q=Q, band=int(np.max(np.abs(np.subtract.outer(*np.nonzero(Qs.toarray() @ Qs.toarray().T))))))
    if sigma is not None:
        d2 = rng.uniform(0.5, 2.0, n)
        mats.append(conj(d2))
        fns.append(Fn(FN_ISQRT_SHIFT, (sigma ** 2, 1.0)))
        meta["d2"] = d2
        meta["sigma"] = sigma
    return _make("planted_sqrt", mats, fns, 175.0, 110.0, 110.0, N, L, seed, meta)


def planted_delay(n=20, seed=5, N=48, L=4, tau=1.0):
    """Diagonal delay NEP a_k - z + b_k exp(-tau z) = 0 (closed form via Lambert W)."""
    rng = np.random.default_rng([12, seed])
    a = np.sort(rng.uniform(1.0, 10.0, n))
    b = rng.uniform(-0.5, 0.5, n)
    mats = [sp.diags(a).tocsr(), -sp.identity(n, format="csr"), sp.diags(b).tocsr()]
    fns = [Fn(FN_CONST), Fn(FN_Z), Fn(FN_EXP_DELAY, (tau,))]
    return _make("planted_delay", mats, fns, 5.5, 4.0, 1.5, N, L, seed, dict(a=a, b=b, tau=tau))


def tiny_qep(n=12, seed=3, N=64, L=4):
    """Random tridiagonal complex QEP K + z C + z^2 M with diagonal M (brute-force pin)."""
    rng = np.random.default_rng([13, seed])
    def tri(scale):
        d = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        e = rng.standard_normal(n - 1) + 1j * rng.standard_normal(n - 1)
        f = rng.standard_normal(n - 1) + 1j * rng.standard_normal(n - 1)
        return sp.diags([f, d, e], [-1, 0, 1]).tocsr() * scale
    K = tri(1.0) + sp.diags(4.0 * np.ones(n))
    C = tri(0.3)
    M = sp.diags(1.0 + rng.random(n)).tocsr()
    return _make("tiny_qep", [K, C, M], [Fn(FN_CONST), Fn(FN_Z), Fn(FN_Z2)],
                 0.0 + 0.0j, 1.6, 1.6, N, L, seed, {})


def loaded_string(n=5000, N=100, L=1):
    """Loaded string rational NEP T1 + z/(z-1) e_n e_n^T - z T3 (Section 7.1, 'String')."""
    e = np.ones(n)
    T1 = sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1], format="lil")
    T1[n - 1, n - 1] = 1.0   # reading: last diagonal 1, which gives the 32 eigenvalues the text states
    T1 = (n * T1).tocsr()
    T3 = sp.diags([e[1:], 4 * e, e[1:]], [-1, 0, 1], format="lil")
    T3[n - 1, n - 1] = 2.0
    T3 = (T3 / (6.0 * n)).tocsr()
    En = sp.csr_matrix(([1.0], ([n - 1], [n - 1])), shape=(n, n))
    # z/(z-1) = p0 z/(z + p1) with p0 = 1, p1 = -1
    return _make("loaded_string", [T1, En, -T3],
                 [Fn(FN_CONST), Fn(FN_RATIONAL, (1.0, -1.0)), Fn(FN_Z)],
                 5001.5, 4998.5, 249.925, N, L, 0, dict(band=1, expected_count=32))


def acoustic_1d(n=1000, N=100, L=2, zeta=1.0):
    """Acoustic-1D QEP z^2 M + z C + K (Section 7.1), C read as (2 pi i / zeta) e_n e_n^T."""
    e = np.ones(n)
    Ks = sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1], format="lil")
    Ks[n - 1, n - 1] = 1.0
    Ks = (n * Ks).tocsr()
    Md = np.ones(n)
    Md[n - 1] = 0.5
    M = sp.diags(-4 * np.pi ** 2 / n * Md).tocsr()
    C = sp.csr_matrix(([2j * np.pi / zeta], ([n - 1], [n - 1])), shape=(n, n))
    return _make("acoustic_1d", [Ks, C, M], [Fn(FN_CONST), Fn(FN_Z), Fn(FN_Z2)],
                 9.9 + 0.8j, 10.1, 1.01, N, L, 0, dict(band=1, expected_count=40))


# --------------------------------------------------------------------------------------
# Distributed-delay NEP, known only by its values: each coupling has its own delay,
#   T(z)_ij = K_ij - z delta_ij + B_ij exp(-tau_ij z),
# so T is not of the form sum_i f_i(z) A_i with few terms (the situation of Section 6, where T
# is a BEM matrix).  K is the unscaled 5-point Laplacian on an s x s grid (spectrum in (0, 8)),
# B and tau symmetric on K's off-diagonal pattern, |B_ij| <= beta, tau_ij ~ U(0.5, 2).
# --------------------------------------------------------------------------------------
def distributed_delay(s=16, N=48, L=4, beta=0.3, gamma=1.507, a=0.53, b=0.1, seed=0):
    """Default contour: the flat ellipse over [0.977, 2.037], whose ends sit in spectral gaps
    of width 0.11 and 0.13; 28 eigenvalues inside (all real: T(x) is real symmetric)."""
    K = grid_laplacian(s, s, 1.0, 1.0)
    n = s * s
    rowptr, colind, kv = _union([K])
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    rng = np.random.default_rng([5, 0])
    lo_ = np.minimum(rows, colind)
    hi_ = np.maximum(rows, colind)
    key = lo_ * n + hi_                     # one draw per unordered pair keeps B, tau symmetric
    uk, inv = np.unique(key, return_inverse=True)
    bvals = beta * rng.uniform(-1.0, 1.0, uk.size)[inv]
    taus = rng.uniform(0.5, 2.0, uk.size)[inv]
    off = rows != colind
    bvals[~off] = 0.0
    diag = (~off).astype(np.float64)
    k0 = kv[0].real.copy()

    def tz(z):
        return k0 - z * diag + bvals * np.exp(-taus * z)

    return TzProblem(name="distributed_delay", n=n, rowptr=rowptr, colind=colind,
                     vals=np.zeros((0, colind.size), dtype=np.complex128), fns=[],
                     gamma=complex(gamma), a=float(a), b=float(b), N=int(N), L=int(L),
                     U=probe_matrix(n, L, seed), seed=seed, meta=dict(s=s, beta=beta), tz=tz)


def by_name(name: str, **kw) -> Problem:
    table = dict(config0=config0, config0_linear=config0_linear, config1=config1,
                 config1b=config1b, config2=config2, planted_sqrt=planted_sqrt,
                 planted_delay=planted_delay, tiny_qep=tiny_qep, loaded_string=loaded_string,
                 acoustic_1d=acoustic_1d, config0_rect=config0_rect, distributed_delay=distributed_delay)
    return table[name](**kw)
