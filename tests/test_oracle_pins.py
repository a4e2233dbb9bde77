"""Pins of the oracle's RSRR (Algorithms 1 and 2) against closed forms, brute force and
values the paper prints.  None of these re-run the oracle's own formulas."""
import json
import os

import numpy as np
import pytest

import oracle as o
import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))


def match(a, b):
    """Pair two eigenvalue lists by minimum-cost bipartite matching; return max rel error."""
    from scipy.optimize import linear_sum_assignment
    a, b = np.asarray(a), np.asarray(b)
    assert a.size == b.size
    if a.size == 0:
        return 0.0
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    return float(np.max(np.abs(a[r] - b[c]) / np.abs(b[c])))


def test_contour_nodes_and_derivative():
    z, dphi, th = o.contour_points(1 + 2j, 3.0, 0.5, 8)
    assert np.allclose(th, 2 * np.pi * (np.arange(8) + 0.5) / 8)
    # trapezoid rule integrates 1/(z - c) exactly enough for interior / exterior c
    for c, expect in [(1 + 2j, 1.0), (1.5 + 2.1j, 1.0), (10 + 0j, 0.0)]:
        z, dphi, _ = o.contour_points(1 + 2j, 3.0, 0.5, 400)
        val = np.sum(dphi / (z - c)) / (1j * 400)
        assert abs(val - expect) < 1e-8


def test_coefficient_branches():
    fns = [w.Fn(w.FN_ISQRT_SHIFT, (0.0, 0.0)), w.Fn(w.FN_ISQRT_SHIFT, (100.0, 1.0)),
           w.Fn(w.FN_EXP_DELAY, (0.7,)), w.Fn(w.FN_RATIONAL, (2.0, -1.0))]
    z = np.array([50 + 10j, 50 - 10j, 150 + 1e-3j])
    F, dF = o.coefficients(fns, z)
    # continued branch agrees with the principal i sqrt(z - s) in the upper half plane
    assert np.allclose(F[0, 1], 1j * np.sqrt(z[0] - 100.0))
    # and is continuous across the real axis left of s (where the principal cut lies)
    F2, _ = o.coefficients(fns, np.array([50 + 1e-9j, 50 - 1e-9j]))
    assert abs(F2[0, 1] - F2[1, 1]) < 1e-6
    # derivatives by central differences
    h = 1e-5
    Fp, _ = o.coefficients(fns, z + h)
    Fm, _ = o.coefficients(fns, z - h)
    assert np.allclose((Fp - Fm) / (2 * h), dF, rtol=1e-6)


def test_vandermonde_rank_pin():
    g = GOLD["vandermonde"]
    lam = np.linspace(g["lo"], g["hi"], g["nodes"])
    ranks_mono, ranks_cheb = [], []
    for Kp in range(10, 101, 5):
        Bm = np.vander(lam, Kp, increasing=True)
        Bc = np.polynomial.chebyshev.chebvander(lam, Kp - 1)
        ranks_mono.append(o.numerical_rank(np.linalg.svd(Bm, compute_uv=False), g["tol"]))
        ranks_cheb.append((Kp, o.numerical_rank(np.linalg.svd(Bc, compute_uv=False), g["tol"])))
    assert max(ranks_mono) <= g["monomial_max_rank"]
    full = [Kp for Kp, r in ranks_cheb if r == g["nodes"]]
    assert g["chebyshev_full_rank_stated"] <= min(full) <= g["chebyshev_full_rank_by"]


def test_linear_laplacian_closed_form():
    """T(z) = K - z I on the 30x30 grid: eigenvalues 4/h^2 (sin^2(i pi h/2) + sin^2(j pi h/2))."""
    p = w.config0_linear()
    h = 1.0 / 31
    k = np.arange(1, 31)
    s = 4 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
    exact = (s[:, None] + s[None, :]).ravel()
    exact = exact[o.inside_contour(exact, p.gamma, p.a, p.b)]
    assert exact.size == 22
    r = o.rsrr(p)
    assert r["lam"].size == 22
    assert match(r["lam"], exact) < 1e-9
    assert r["resid_scaled"].max() < 1e-10


def test_tiny_qep_companion_brute_force():
    p = w.tiny_qep()
    K, C, M = (p.term(i).toarray() for i in range(3))
    n = p.n
    A = np.block([[np.zeros((n, n)), np.eye(n)], [-K, -C]])
    B = np.block([[np.eye(n), np.zeros((n, n))], [np.zeros((n, n)), M]])
    ev = np.linalg.eigvals(np.linalg.solve(B, A))
    inside = ev[o.inside_contour(ev, p.gamma, p.a, p.b)]
    r = o.rsrr(p, N_S=500, K=4)
    assert r["lam"].size == inside.size > 0
    assert match(r["lam"], inside) < 1e-9
    assert r["resid"].max() < 1e-10


def test_planted_sqrt_closed_form():
    """d0 - z + i d1 sqrt(z) = 0  <=>  w^2 - i d1 w - d0 = 0, w = sqrt(z), Re w > 0."""
    p = w.planted_sqrt()
    d0, d1 = p.meta["d0"], p.meta["d1"]
    wr = (1j * d1 + np.sqrt(4 * d0 - d1 ** 2 + 0j)) / 2
    exact = wr ** 2
    exact = exact[o.inside_contour(exact, p.gamma, p.a, p.b)]
    r = o.rsrr(p)
    assert r["lam"].size == exact.size > 5
    assert match(r["lam"], exact) < 1e-9
    assert r["resid"].max() < 1e-10


def test_planted_sqrt_continued_branch():
    """Adds -sqrt(sigma^2 - z) d2: scalar roots by Newton, counted by the argument principle."""
    sigma = 18.0
    p = w.planted_sqrt(sigma=sigma)
    d0, d1, d2 = p.meta["d0"], p.meta["d1"], p.meta["d2"]
    s2 = sigma ** 2

    def f(z, k):
        return d0[k] - z + 1j * d1[k] * np.sqrt(z) - d2[k] * np.sqrt(s2 - z)

    def df(z, k):
        return -1 + 0.5j * d1[k] / np.sqrt(z) + 0.5 * d2[k] / np.sqrt(s2 - z)

    zc, dphi, _ = o.contour_points(p.gamma, p.a, p.b, 4000)
    roots = []
    for k in range(p.n):
        cnt = np.sum(df(zc, k) / f(zc, k) * dphi) / (1j * 4000)
        assert abs(cnt - round(cnt.real)) < 1e-6 and round(cnt.real) in (0, 1)
        if round(cnt.real) == 1:
            z = complex(d0[k])
            for _ in range(60):
                z = z - f(z, k) / df(z, k)
            assert abs(f(z, k)) < 1e-10 * abs(z)
            roots.append(z)
    r = o.rsrr(p)
    assert r["lam"].size == len(roots) > 5
    assert match(r["lam"], roots) < 1e-9


def test_planted_delay_lambert_w():
    """a - z + b exp(-tau z) = 0  <=>  z = a + W(b tau exp(-a tau)) / tau."""
    from scipy.special import lambertw
    p = w.planted_delay()
    a, b, tau = p.meta["a"], p.meta["b"], p.meta["tau"]
    roots = []
    for br in range(-3, 4):
        roots.append(a + lambertw(b * tau * np.exp(-a * tau), br) / tau)
    roots = np.concatenate(roots)
    exact = roots[o.inside_contour(roots, p.gamma, p.a, p.b)]
    r = o.rsrr(p)
    assert r["lam"].size == exact.size > 5
    assert match(r["lam"], exact) < 1e-9


def test_loaded_string_count_printed():
    g = GOLD["loaded_string"]
    p = w.loaded_string(n=g["n"], N=g["N"], L=g["L"])
    assert (p.gamma, p.a, p.b) == (g["gamma"], g["a"], g["b"])
    r = o.rsrr(p, N_S=g["N_S"], K=g["K"])
    assert r["lam"].size == g["count"]
    assert np.all((r["lam"].real > g["interval"][0]) & (r["lam"].real < g["interval"][1]))
    assert r["resid_scaled"].max() < 1e-10


def test_acoustic_1d_count_printed():
    g = GOLD["acoustic_1d"]
    p = w.acoustic_1d(n=g["n"], N=g["N"], L=g["L"])
    r = o.rsrr(p, N_S=g["N_S"], K=g["K"])
    assert r["lam"].size == g["count"]
    assert r["resid_scaled"].max() < 1e-10


def test_moment_span_inclusion():
    """M_hat = S_hat D Z (Eq. eq-hatMS): quadrature moments lie in span(S) (Eq. eq-setsMS)."""
    p = w.config0_linear(N=16, L=4, nx=12, ny=10)
    Shat, _, _ = o.sample(p)
    S, sigma, k = o.truncated_basis(Shat, 1e-14)
    z, dphi, _ = o.contour_points(p.gamma, p.a, p.b, p.N)
    omega = dphi / (1j * p.N)
    for al in range(6):
        Mh = sum(omega[i] * z[i] ** al * Shat[:, i * p.L:(i + 1) * p.L] for i in range(p.N))
        res = Mh - S @ (S.conj().T @ Mh)
        assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(Mh)


def test_sample_backward_error_and_dense_path_agree():
    p = w.config0(N=8, L=3, nx=9, ny=7)
    Sb, infos, eta = o.sample(p)
    Sd, _, eta_d = o.sample(p, dense=True)
    assert np.all(infos == 0)
    assert eta.max() < 1e-14 and eta_d.max() < 1e-14
    assert np.allclose(Sb, Sd, rtol=1e-10, atol=1e-13 * np.abs(Sd).max())


def test_config0_counts_and_residuals():
    """Config 0: 22 eigenvalues inside (argument principle on det T, oracle-independent
    of the subspace), residual scaled <= 1e-10."""
    p = w.config0()
    r = o.rsrr(p)
    assert r["lam"].size == 22
    assert r["resid_scaled"].max() < 1e-10


def test_config1_small_has_no_eigenvalues_inside():
    """Damped QEP with the config-1 contour: every eigenvalue with Re >= -2.5 has Im < 10
    (closed form via the pencil K v = mu M v), so the count is 0."""
    p = w.config1(s=12, N=16, L=4)
    z = w.problems.damped_eigs(12, 144)
    assert not np.any(o.inside_contour(z, p.gamma, p.a, p.b))
    assert not np.any(o.inside_contour(np.conj(z), p.gamma, p.a, p.b))
    r = o.rsrr(p, N_S=200)
    assert r["lam"].size == 0


def test_config1b_small_closed_form():
    p = w.config1b(s=20, N=32, L=8)
    exact = w.problems.damped_eigs(20, 400)
    exact = np.concatenate([exact, exact.conj()])
    exact = exact[o.inside_contour(exact, p.gamma, p.a, p.b)]
    assert exact.size >= 8
    r = o.rsrr(p, N_S=500)
    assert r["lam"].size == exact.size
    assert match(r["lam"], exact) < 1e-9


@pytest.mark.parametrize("s,idx", [(8, 0), (10, 2), (12, 0)])
def test_config3_shape_linear_case_matches_eig(s, idx):
    """Time-delay batch member with tau = 0: T(z) = -zI + A0 + A1 is linear, so its eigenvalues
    are those of A0 + A1 (numpy eig, dense); the oracle's dense path must find exactly the ones
    inside the circle."""
    p = w.config3_member(idx, s=s, N=32, L=8, tau=0.0)
    ev = np.linalg.eigvals(p.term(1).toarray() + p.term(2).toarray())
    inside = ev[o.inside_contour(ev, p.gamma, p.a, p.b)]
    r = o.rsrr(p, dense=True)
    assert r["lam"].size == inside.size > 0
    assert match(r["lam"], inside) < 1e-9


@pytest.mark.parametrize("s,idx", [(8, 0), (10, 2)])
def test_config3_member_count_and_perturbation_bound(s, idx):
    """Time-delay member (tau > 0): on the circle Re z > 30, so e^{-tau z} A1 is a tiny
    perturbation of A0 and (Bauer-Fike, A0 symmetric) every eigenvalue lies within
    |e^{-tau lambda}| ||A1||_2 of a closed-form Laplacian level; the count inside equals the
    number of levels (with multiplicity) inside."""
    p = w.config3_member(idx, s=s, N=32, L=8)
    h = 1.0 / (s + 1)
    l1 = 4.0 / h ** 2 * np.sin(np.arange(1, s + 1) * np.pi * h / 2) ** 2
    mu = (l1[:, None] + l1[None, :]).ravel().astype(complex)
    count = int(np.count_nonzero(o.inside_contour(mu, p.gamma, p.a, p.b)))
    r = o.rsrr(p, dense=True)
    assert r["lam"].size == count > 0
    bound = np.abs(np.exp(-p.meta["tau"] * r["lam"])) * np.linalg.norm(p.term(2).toarray(), 2)
    dist = np.min(np.abs(r["lam"][:, None] - mu[None, :]), axis=1)
    assert np.all(dist <= bound * (1 + 1e-6) + 1e-9)
    assert r["resid_scaled"].max() < 1e-10


def test_moment_scheme_closed_form():
    """SSRR moment scheme (Eqs. eq-malpha-qud, eq-hatM) on T = K - zI: with K' = N the moments span
    the same space as the samples (Eq. eq-hatMS with Z invertible), and for K' = N and smaller K'
    the eigenvalues are the closed-form Laplacian ones inside the circle."""
    p = w.config0_linear(N=32, L=16)
    h = 1.0 / 31
    k = np.arange(1, 31)
    lam1 = 4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
    mu = (lam1[:, None] + lam1[None, :]).ravel().astype(complex)
    exact = mu[o.inside_contour(mu, p.gamma, p.a, p.b)]
    samp = o.rsrr(p)
    for Kp in (32, 12):
        r = o.rsrr(p, moments=Kp)
        assert r["lam"].size == exact.size == 22
        assert match(r["lam"], exact) < 1e-9
        if Kp == p.N:
            assert r["k_S"] == samp["k_S"]
        else:
            assert r["k_S"] < samp["k_S"]


def test_interior_sampling_points_closed_form():
    """Sampling at points that are not the contour's nodes (Section 3.2: any points of the domain
    serve, the ones inside the contour included): the samples solve T(z_j) X_j = U at the given
    points, and the eigenvalues inside the ellipse are still the closed-form Laplacian ones."""
    p = w.config0_linear(N=32, L=16)
    assert [f.kind for f in p.fns] == [w.FN_CONST, w.FN_Z]
    h = 1.0 / 31
    lam1 = 4.0 / h ** 2 * np.sin(np.arange(1, 31) * np.pi * h / 2) ** 2
    mu = (lam1[:, None] + lam1[None, :]).ravel().astype(complex)
    exact = mu[o.inside_contour(mu, p.gamma, p.a, p.b)]
    rng = np.random.default_rng(5)
    r, ph = np.sqrt(rng.uniform(0, 0.8, 32)), rng.uniform(0, 2 * np.pi, 32)
    z = p.gamma + r * (p.a * np.cos(ph) + 1j * p.b * np.sin(ph))
    Shat, infos, eta = o.sample(p, z=z)
    for j in (0, 7, 31):
        T = p.term(0) + z[j] * p.term(1)
        X = Shat[:, j * p.L:(j + 1) * p.L]
        assert np.linalg.norm(T @ X - p.U) < 1e-12 * np.linalg.norm(p.U)
    res = o.rsrr(p, z=z)
    assert res["lam"].size == exact.size == 22
    assert match(res["lam"], exact) < 1e-9


def test_sampling_scheme_outranks_moment_scheme_on_string():
    """Sections 3.1 and 6.1: with high-order moments M_hat becomes numerically rank deficient
    while S_hat keeps a clear gap after the eigenvalue count.  On the loaded string (L = 1,
    N = 100, the paper's contour, K' = N) the 32nd singular value of M_hat sits at the rounding
    floor, that of S_hat two decades below sigma_1, and the moment scheme's eigenpairs are
    orders of magnitude less accurate, as the paper's residual plots show."""
    G = GOLD["loaded_string"]
    p = w.by_name("loaded_string", n=G["n"], N=G["N"], L=G["L"])
    r = o.rsrr(p, N_S=G["N_S"], K=G["K"])
    rm = o.rsrr(p, N_S=G["N_S"], K=G["K"], moments=G["N"])
    c = G["count"]
    assert r["lam"].size == rm["lam"].size == c
    assert r["sigma"][c - 1] / r["sigma"][0] > 1e-4
    assert rm["sigma"][c - 1] / rm["sigma"][0] < 1e-9
    assert r["k_S"] > rm["k_S"]
    assert r["resid_scaled"].max() < 1e-10
    assert rm["resid_scaled"].max() > 1e3 * r["resid_scaled"].max()


def test_rectangle_rule():
    """The rectangle's Gauss-Legendre rule (Section 7.2, the gun example): each side's m-point
    rule integrates t^k exactly for k < 2m, so the contour integral of any polynomial of
    degree < 2 min(m) vanishes; the Cauchy integral of 1/(z - c) is 1 inside, 0 outside
    (counter-clockwise orientation); the paper's "10-5" split for N = 30."""
    for m in (1, 5, 10, 51):
        t, om = np.polynomial.legendre.leggauss(m)
        for k in range(2 * m):
            assert abs(om @ t ** k - (2.0 / (k + 1) if k % 2 == 0 else 0.0)) < 1e-14
    g, a, b = 237.7 + 20j, 97.7, 25.0
    assert o.rectangle_split(30, a, b, 10) == (10, 5)
    assert o.rectangle_split(36, a, b, 12) == (12, 6)
    assert o.rectangle_split(500, a, b) == (199, 51)
    z, wq = o.contour_rule(g, a, b, 30, "rectangle", 10)
    d = z - g
    on_side = np.minimum(np.abs(np.abs(d.real) - a), np.abs(np.abs(d.imag) - b))
    assert z.size == 30 and on_side.max() < 1e-12 * a
    assert np.allclose(z[:10].imag, g.imag - b) and np.all(np.diff(z[:10].real) > 0)  # bottom, left to right
    u = (z - g) / a
    for k in range(10):
        assert abs(wq @ u ** k) < 1e-13
    z, wq = o.contour_rule(g, a, b, 400, "rectangle")
    for c, want in ((g, 1.0), (g + 50 - 10j, 1.0), (g + 150, 0.0), (g + 60j, 0.0)):
        assert abs(wq @ (1.0 / (z - c)) - want) < 1e-10
    # the ellipse's rule is the trapezoid one of Eq. eq-Ap-num
    z, wq = o.contour_rule(1 + 2j, 3.0, 0.5, 256)
    ze, dphi, _ = o.contour_points(1 + 2j, 3.0, 0.5, 256)
    assert np.allclose(z, ze) and np.allclose(wq, dphi / (256j))
    assert abs(wq @ (1.0 / (z - (1.5 + 2.1j))) - 1) < 1e-12


def test_rectangle_contour_closed_form():
    """RSRR with the rectangle contour and Gauss-Legendre sampling points: on T = K - zI the
    eigenvalues inside the rectangle are the closed-form Laplacian ones, the winding number
    counts them, and on the gun-like NEP the rectangle finds the same eigenvalues as the
    ellipse run inside the rectangle."""
    p = w.config0_rect(linear=True)
    h = 1.0 / 31
    lam1 = 4.0 / h ** 2 * np.sin(np.arange(1, 31) * np.pi * h / 2) ** 2
    mu = (lam1[:, None] + lam1[None, :]).ravel().astype(complex)
    exact = mu[o.inside_contour(mu, p.gamma, p.a, p.b, "rectangle")]
    r = o.rsrr(p)
    assert r["lam"].size == exact.size == 14
    assert r["n_winding"] == 14 and abs(r["winding"] - 14) < 1e-6
    assert match(r["lam"], exact) < 1e-9
    q = w.config0_rect()
    rq = o.rsrr(q)
    re = o.rsrr(w.config0())
    ref = re["lam"][o.inside_contour(re["lam"], q.gamma, q.a, q.b, "rectangle")]
    assert rq["lam"].size == ref.size == 14
    assert match(rq["lam"], ref) < 1e-9
    assert rq["resid_scaled"].max() < 1e-10


def test_chebyshev_kind():
    """The Chebyshev function kind: tau_m(cos t) = cos(m t) and tau_m'(cos t) = m sin(m t)/sin t,
    on an interval [lo, hi] mapped to [-1, 1]."""
    lo, hi = 100.0, 400.0
    t = np.linspace(0.1, 3.0, 7)
    z = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(t)
    for m in (0, 1, 2, 7, 30):
        F, dF = o.coefficients([w.Fn(w.FN_CHEBYSHEV, (m, lo, hi))], z)
        assert np.allclose(F[:, 0], np.cos(m * t), atol=1e-12)
        assert np.allclose(dF[:, 0], m * np.sin(m * t) / np.sin(t) * 2.0 / (hi - lo), atol=1e-10)


def test_chebyshev_interpolant_reproduces_polynomial_nep():
    """Section 6.2: a degree-d Chebyshev interpolant reproduces any T of degree <= d, so for the
    quadratic NEP the reduced interpolant equals sum_i f_i(z) P_i at any z when d >= 2 (and not
    for d = 1), and the eigenvalues are the companion linearisation's.  This decides the j = 0
    weight: with the constant term not halved the d = 2 interpolant misses by P_hat_0."""
    p = w.tiny_qep()
    Shat, _, _ = o.sample(p)
    S, _, _ = o.truncated_basis(Shat, 1e-14)
    P = o.project(p, S)
    lo, hi = p.gamma.real - p.a, p.gamma.real + p.a
    rng = np.random.default_rng(7)
    zs = rng.normal(size=5) * 2 + 1j * rng.normal(size=5)
    F, _ = o.coefficients(p.fns, zs)
    for d, exact in ((1, False), (2, True), (5, True)):
        Ph, fns = o.chebyshev_reduce(p, S, d, lo, hi)
        Fc, _ = o.coefficients(fns, zs)
        err = max(np.linalg.norm(np.tensordot(Fc[t], Ph, 1) - np.tensordot(F[t], P, 1)) /
                  np.linalg.norm(np.tensordot(F[t], P, 1)) for t in range(zs.size))
        assert (err < 1e-12) == exact
    K, C, M = (p.term(i).toarray() for i in range(3))
    n = p.n
    A = np.block([[np.zeros((n, n)), np.eye(n)], [-K, -C]])
    B = np.block([[np.eye(n), np.zeros((n, n))], [np.zeros((n, n)), M]])
    ev = np.linalg.eigvals(np.linalg.solve(B, A))
    ev = ev[o.inside_contour(ev, p.gamma, p.a, p.b)]
    r = o.rsrr(p, K=4, chebyshev=(2, lo, hi))
    assert r["lam"].size == ev.size > 0
    assert match(r["lam"], ev) < 1e-9


def test_chebyshev_route_converges_on_sqrt_nep():
    """Section 6.2: for T holomorphic near the interval the interpolant's error decays
    exponentially in d.  Gun-like sqrt NEP (branch points at 0 and 108.8^2), flat ellipse
    (250; 150, 10) around the interval [100, 400]: d = 10 and d = 20 approach the eigenvalues of
    the direct reduced NEP geometrically; residuals are judged on the true T."""
    q = w.config0()
    q.b = 10.0
    ref = o.rsrr(q)
    errs = []
    for d in (10, 20):
        r = o.rsrr(q, chebyshev=(d, 100.0, 400.0))
        assert r["lam"].size == ref["lam"].size == 22
        errs.append(match(r["lam"], ref["lam"]))
        assert r["resid_scaled"].max() < (1e-10 if d == 20 else 1e-8)
    assert errs[0] < 1e-8 and errs[1] < 1e-13 and errs[1] < 1e-3 * errs[0]


def test_tz_route_equals_affine_route():
    """A NEP given by its values T(z) (no affine form; Section 6) goes through the same steps:
    built from config 0's sum_i f_i(z) A_i it yields the same samples and the same Chebyshev
    eigenvalues as the affine description."""
    p = w.config0()
    p.b = 10.0
    F = lambda z: o.coefficients(p.fns, np.array([z]))[0][0]
    q = w.TzProblem(name="config0_tz", n=p.n, rowptr=p.rowptr, colind=p.colind,
                    vals=np.zeros((0, p.nnz), np.complex128), fns=[], gamma=p.gamma, a=p.a, b=p.b,
                    N=p.N, L=p.L, U=p.U, tz=lambda z: F(z) @ p.vals)
    Sp, _, _ = o.sample(p)
    Sq, _, _ = o.sample(q)
    assert np.abs(Sp - Sq).max() <= 1e-13 * np.abs(Sp).max()
    rp = o.rsrr(p, chebyshev=(16, 100.0, 400.0))
    rq = o.rsrr(q, chebyshev=(16, 100.0, 400.0))
    assert rq["lam"].size == rp["lam"].size == 22
    assert match(rq["lam"], rp["lam"]) < 1e-12


def test_distributed_delay_count_by_argument_principle():
    """The distributed-delay NEP (one delay per coupling, known only by its values): the count
    inside the contour from the argument principle on det T(z) (dense log-determinants along
    the ellipse, independent of the method) is the Chebyshev route's count, and each
    eigenvalue makes T(lambda) singular to working accuracy."""
    p = w.distributed_delay()
    th = 2 * np.pi * (np.arange(3000) + 0.5) / 3000
    zc = p.gamma + p.a * np.cos(th) + 1j * p.b * np.sin(th)
    def logdet(z):
        T = np.zeros((p.n, p.n), np.complex128)
        T[np.repeat(np.arange(p.n), np.diff(p.rowptr)), p.colind] = p.tz(z)
        sgn, ld = np.linalg.slogdet(T)
        return np.angle(sgn)
    ph = np.unwrap([logdet(z) for z in zc])
    count = int(np.rint((ph[-1] - ph[0] + (ph[1] - ph[0])) / (2 * np.pi)))
    r = o.rsrr(p, chebyshev=(16, p.gamma.real - p.a, p.gamma.real + p.a))
    assert count == r["lam"].size == 28
    for lam in r["lam"][:5]:
        T = np.zeros((p.n, p.n), np.complex128)
        T[np.repeat(np.arange(p.n), np.diff(p.rowptr)), p.colind] = p.tz(lam)
        sv = np.linalg.svd(T, compute_uv=False)
        assert sv[-1] < 1e-12 * sv[0]
