"""Parity of rsrr_project (Algorithm 2 Step 3, Eq. eq-Zs-expr) and rsrr_solve (Algorithm 1,
Algorithm 2 Step 5) with the oracle, closed forms and the paper's printed counts.

Bars: eigenvalues to relative 1e-9 (matched by minimum-cost assignment), the same count, and
scaled residuals ||T(l) v|| / sum_i |f_i(l)| ||A_i||_F <= 1e-10 (the raw residual's FP64 floor
u ||T(l)|| exceeds 1e-10 on the grid problems, whose K is scaled by 1/h^2)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as w
from gpu_util import match, open_nep, rel_err_cols

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def gpu_rsrr(rs, prob, precision=None, tol=1e-12, N_S=500, K=2, delta=1e-14):
    precision = rs.RSRR_FP64 if precision is None else precision
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, precision, tol, 12)
    Shat = h.samples()
    kS = h.project(delta)
    S, P, sig = h.basis(), h.projected(), h.sigma()
    lam, V, res = h.solve(N_S, K, 1e3, 4096, True)
    info = h.info()
    hs = h.hankel_sigma(K)
    h.close()
    return dict(Shat=Shat, kS=kS, S=S, P=P, sigma=sig, lam=lam, V=V, resid=res, info=info, sigma_H=hs)


def scaled(prob, lam, raw):
    F, _ = oracle.coefficients(prob.fns, lam)
    nA = np.array([np.linalg.norm(prob.vals[i]) for i in range(prob.J)])
    return raw / (np.abs(F) @ nA)


def near_threshold(sigma, delta):
    s = np.asarray(sigma)
    return int(np.sum((s > 0.1 * delta * s[0]) & (s < 10 * delta * s[0])))


def check_projection(rs, prob, g, delta=1e-14):
    ref_S, ref_sig, ref_k = oracle.truncated_basis(g["Shat"], delta)
    S = g["S"]
    # S orthonormal, captures S_hat down to the truncation level, same rank up to near-ties
    assert np.linalg.norm(S.conj().T @ S - np.eye(g["kS"])) < 1e-12
    resid = np.linalg.norm(g["Shat"] - S @ (S.conj().T @ g["Shat"]), 2)
    assert resid <= 20 * delta * ref_sig[0] + 1e-15 * np.linalg.norm(g["Shat"])
    assert abs(g["kS"] - ref_k) <= near_threshold(ref_sig, delta)
    top = ref_sig[ref_sig > 1e-6 * ref_sig[0]]
    assert np.allclose(g["sigma"][:top.size], top, rtol=1e-9, atol=1e-13 * ref_sig[0])
    # P_i = S^H A_i S against the oracle's projection of the same basis
    assert np.allclose(g["P"], oracle.project(prob, S), rtol=0, atol=1e-11 * np.abs(g["P"]).max())


CLOSED = ["config0_linear", "tiny_qep", "planted_sqrt", "planted_delay"]


def exact_eigs(name, prob):
    if name == "config0_linear":
        h = 1.0 / 31
        s = 4 / h ** 2 * np.sin(np.arange(1, 31) * np.pi * h / 2) ** 2
        ev = (s[:, None] + s[None, :]).ravel()
    elif name == "tiny_qep":
        K, C, M = (prob.term(i).toarray() for i in range(3))
        n = prob.n
        A = np.block([[np.zeros((n, n)), np.eye(n)], [-K, -C]])
        B = np.block([[np.eye(n), np.zeros((n, n))], [np.zeros((n, n)), M]])
        ev = np.linalg.eigvals(np.linalg.solve(B, A))
    elif name == "planted_sqrt":
        d0, d1 = prob.meta["d0"], prob.meta["d1"]
        ev = ((1j * d1 + np.sqrt(4 * d0 - d1 ** 2 + 0j)) / 2) ** 2
    else:
        from scipy.special import lambertw
        a, b, tau = prob.meta["a"], prob.meta["b"], prob.meta["tau"]
        ev = np.concatenate([a + lambertw(b * tau * np.exp(-a * tau), k) / tau for k in range(-3, 4)])
    return ev[oracle.inside_contour(ev, prob.gamma, prob.a, prob.b)]


@pytest.mark.parametrize("name", CLOSED)
def test_eigenvalues_match_closed_form(rs, name):
    prob = w.by_name(name)
    K = 4 if name == "tiny_qep" else 2
    g = gpu_rsrr(rs, prob, K=K)
    ex = exact_eigs(name, prob)
    assert g["lam"].size == ex.size > 0
    assert match(g["lam"], ex) < 1e-9
    assert scaled(prob, g["lam"], g["resid"]).max() < 1e-10
    check_projection(rs, prob, g)


@pytest.mark.parametrize("name,kw,NS,K", [
    ("config0", dict(), 500, 2),
    ("loaded_string", dict(n=GOLD["loaded_string"]["n"], N=GOLD["loaded_string"]["N"], L=1), 1000, 8),
    ("acoustic_1d", dict(), 1000, 2),
])
def test_eigenvalues_match_oracle(rs, name, kw, NS, K):
    prob = w.by_name(name, **kw)
    ref = oracle.rsrr(prob, N_S=NS, K=K)
    g = gpu_rsrr(rs, prob, N_S=NS, K=K)
    assert g["lam"].size == ref["lam"].size
    assert match(g["lam"], ref["lam"]) < 1e-9
    assert scaled(prob, g["lam"], g["resid"]).max() < 1e-10
    # eigenvectors: same residual level, and v_gpu spans the oracle's v per simple eigenvalue
    for t in range(min(5, g["lam"].size)):
        j = np.argmin(np.abs(ref["lam"] - g["lam"][t]))
        c = abs(np.vdot(ref["V"][:, j], g["V"][:, t]))
        assert c > 1 - 1e-6
    check_projection(rs, prob, g)
    if name == "loaded_string":
        assert g["lam"].size == GOLD["loaded_string"]["count"]
    if name == "acoustic_1d":
        assert g["lam"].size == GOLD["acoustic_1d"]["count"]


def test_mixed_precision_pipeline_matches_fp64(rs):
    prob = w.config0()
    g64 = gpu_rsrr(rs, prob)
    gmx = gpu_rsrr(rs, prob, precision=rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, tol=1e-10)
    assert gmx["info"]["refine_sweeps"] >= 1
    assert gmx["lam"].size == g64["lam"].size == 22
    assert match(gmx["lam"], g64["lam"]) < 1e-9
    assert scaled(prob, gmx["lam"], gmx["resid"]).max() < 1e-10


def test_config1_contour_encloses_nothing(rs):
    prob = w.config1(s=16, N=16, L=4)
    g = gpu_rsrr(rs, prob, N_S=200)
    assert g["lam"].size == 0
    assert g["info"]["n_winding"] == 0


def test_config1b_closed_form(rs):
    prob = w.config1b(s=20, N=32, L=8)
    exact = w.problems.damped_eigs(20, 400)
    exact = np.concatenate([exact, exact.conj()])
    exact = exact[oracle.inside_contour(exact, prob.gamma, prob.a, prob.b)]
    g = gpu_rsrr(rs, prob, precision=rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, tol=1e-10)
    assert g["lam"].size == exact.size
    assert match(g["lam"], exact) < 1e-9
    assert scaled(prob, g["lam"], g["resid"]).max() < 1e-10


def test_hankel_singular_values_match_oracle(rs):
    prob = w.planted_sqrt()
    g = gpu_rsrr(rs, prob)
    ref = oracle.rsrr(prob)
    P = g["P"]
    lam, gg, diag = oracle.reduced_ss(P, prob.fns, prob.gamma, prob.a, prob.b, 500, 2, 1e3, return_diag=True)
    sH = diag["sigma_H"]
    top = sH > 1e-8 * sH[0]
    assert np.allclose(g["sigma_H"][top], sH[top], rtol=1e-8)
    assert g["info"]["n_winding"] == diag["n_winding"]
    assert abs(complex(g["info"]["winding_re"], g["info"]["winding_im"]) - diag["winding"]) < 1e-8
    assert ref["lam"].size == g["lam"].size


def test_callback_function_kind_matches_builtin(rs):
    """RSRR_F_CALLBACK: the same NEP with its z^2 (quadratic) and i sqrt(z) (planted sqrt) terms
    supplied as host callbacks gives the built-in kinds' eigenvalues."""
    import cmath
    for name, K in (("tiny_qep", 4), ("planted_sqrt", 2)):
        prob = w.by_name(name)
        builtin = gpu_rsrr(rs, prob, K=K)
        fns = []
        for f in prob.fns:
            if f.kind == w.FN_Z2:
                fns.append(rs.callback_fn(lambda z: z * z, lambda z: 2 * z))
            elif f.kind == w.FN_ISQRT_SHIFT and f.params()[1] == 0.0:
                s = f.params()[0]
                fns.append(rs.callback_fn(lambda z, s=s: 1j * cmath.sqrt(z - s),
                                          lambda z, s=s: 0.5j / cmath.sqrt(z - s)))
            else:
                fns.append((f.kind, f.params()))
        assert any(k == rs.F_CALLBACK for k, _ in fns)
        h = rs.Nep(prob.n, prob.rowptr, prob.colind, prob.vals, fns)
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12)
        h.project(1e-14)
        lam, V, res = h.solve(500, K, 1e3, 4096, True)
        assert lam.size == builtin["lam"].size > 0
        assert match(lam, builtin["lam"]) < 1e-12
        h.close()


@pytest.mark.parametrize("name,Kp", [("config0_linear", 32), ("config0_linear", 12), ("config0", 16)])
def test_moment_scheme_matches_oracle(rs, name, Kp):
    """rsrr_project_moments (SSRR moment scheme, Eqs. eq-malpha-qud, eq-hatMS) on the device
    against the oracle's moment scheme on the same samples: the truncation of M_hat, the
    projected matrices and the eigenvalues."""
    prob = w.by_name(name)
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
    Shat = h.samples()
    kS = h.project_moments(Kp)
    assert h.info()["proj_cols"] == Kp * prob.L
    S, P, sig = h.basis(), h.projected(), h.sigma()
    lam, V, res = h.solve(500, 2, 1e3, 4096, True)
    h.close()
    M = oracle.moment_matrix(prob, Shat, Kp)
    ref_S, ref_sig, ref_k = oracle.truncated_basis(M, 1e-14)
    assert abs(kS - ref_k) <= near_threshold(ref_sig, 1e-14)
    assert np.linalg.norm(S.conj().T @ S - np.eye(kS)) < 1e-12
    resid = np.linalg.norm(M - S @ (S.conj().T @ M), 2)
    assert resid <= 20 * 1e-14 * ref_sig[0] + 1e-15 * np.linalg.norm(M)
    top = ref_sig[ref_sig > 1e-6 * ref_sig[0]]
    assert np.allclose(sig[:top.size], top, rtol=1e-9, atol=1e-13 * ref_sig[0])
    assert np.allclose(P, oracle.project(prob, S), rtol=0, atol=1e-11 * np.abs(P).max())
    ref = oracle.rsrr(prob, moments=Kp)
    assert lam.size == ref["lam"].size > 0
    assert match(lam, ref["lam"]) < 1e-9
    if name == "config0_linear":
        assert match(lam, exact_eigs(name, prob)) < 1e-9


def interior_points(prob, N, seed=5, rmax=0.8):
    rng = np.random.default_rng(seed)
    r, ph = np.sqrt(rng.uniform(0, rmax, N)), rng.uniform(0, 2 * np.pi, N)
    return prob.gamma + r * (prob.a * np.cos(ph) + 1j * prob.b * np.sin(ph))


@pytest.mark.parametrize("name,prec", [("config0_linear", "fp64"), ("config0", "c64"), ("tiny_qep", "fp64")])
def test_sample_points_matches_oracle(rs, name, prec):
    """rsrr_sample_points (Section 3.2: sampling points anywhere in the domain): samples at interior
    points equal the oracle's solves at the same points, and the eigenvalues inside the ellipse
    equal the oracle's (and the closed form where there is one)."""
    prob = w.by_name(name)
    z = interior_points(prob, prob.N)
    mode = rs.RSRR_FP64 if prec == "fp64" else rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL
    h = open_nep(rs, prob)
    h.sample_points(prob.gamma, prob.a, prob.b, z, prob.L, prob.U, mode, 1e-12 if prec == "fp64" else 1e-10, 20)
    X = h.samples()
    ref, infos, _ = oracle.sample(prob, z=z)
    assert np.all(infos == 0)
    assert rel_err_cols(X, ref).max() < 1e-8
    with pytest.raises(rs.RsrrError) as e:
        h.project_moments(4)
    assert e.value.name == "EINVAL"
    h.project(1e-14)
    K = 4 if name == "tiny_qep" else 2
    lam, V, res = h.solve(500, K, 1e3, 4096, True)
    h.close()
    refr = oracle.rsrr(prob, K=K, z=z)
    assert lam.size == refr["lam"].size > 0
    assert match(lam, refr["lam"]) < 1e-9
    assert scaled(prob, lam, res).max() < 1e-10
    if name in CLOSED:
        assert match(lam, exact_eigs(name, prob)) < 1e-9


def test_sample_points_at_contour_nodes_equals_sample(rs):
    """With the contour's own trapezoid nodes, rsrr_sample_points gives rsrr_sample's samples."""
    prob = w.config0()
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
    X0 = h.samples()
    th = 2 * np.pi * (np.arange(prob.N) + 0.5) / prob.N
    z = prob.gamma + prob.a * np.cos(th) + 1j * prob.b * np.sin(th)
    h.sample_points(prob.gamma, prob.a, prob.b, z, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
    assert rel_err_cols(h.samples(), X0).max() < 1e-13
    with pytest.raises(rs.RsrrError) as e:
        h.sample_points(prob.gamma, prob.a, prob.b, np.array([np.nan]), prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
    assert e.value.name == "EINVAL"
    h.close()


def test_sampling_vs_moment_scheme_on_string(rs):
    """The paper's comparison (Sections 3.1, 6.1) on the device: on the loaded string with K' = N
    the device's M_hat is numerically rank deficient where S_hat is not, the truncation of each
    matches the oracle's, and the moment scheme's eigenpairs are far less accurate."""
    G = GOLD["loaded_string"]
    prob = w.by_name("loaded_string", n=G["n"], N=G["N"], L=G["L"])
    out = {}
    for Kp in (0, G["N"]):
        h = open_nep(rs, prob)
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
        Shat = h.samples()
        kS = h.project_moments(Kp) if Kp else h.project(1e-14)
        sig = h.sigma()
        lam, V, res = h.solve(G["N_S"], G["K"], 1e3, 4096, True)
        h.close()
        M = oracle.moment_matrix(prob, Shat, Kp) if Kp else Shat
        _, ref_sig, ref_k = oracle.truncated_basis(M, 1e-14)
        assert abs(kS - ref_k) <= near_threshold(ref_sig, 1e-14)
        out[Kp] = (kS, sig, lam, scaled(prob, lam, res))
    c = G["count"]
    (k0, s0, l0, r0), (k1, s1, l1, r1) = out[0], out[G["N"]]
    assert l0.size == l1.size == c
    assert s0[c - 1] / s0[0] > 1e-4 and s1[c - 1] / s1[0] < 1e-9
    assert k0 > k1
    assert r0.max() < 1e-10 and r1.max() > 1e3 * r0.max()


def sample_rect(rs, prob, h, precision=None, tol=1e-12):
    precision = rs.RSRR_FP64 if precision is None else precision
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, precision, tol, 20,
             shape=rs.RSRR_CONTOUR_RECTANGLE, side_nodes=prob.side_nodes)


@pytest.mark.parametrize("linear", [True, False])
def test_rectangle_contour_matches_oracle(rs, linear):
    """Rectangle contour with Gauss-Legendre points ("10-5", Section 7.2): the samples at the
    rule's nodes, the winding number, the eigenvalues (closed form for T = K - zI) and the
    residuals against the oracle's run on the same rectangle."""
    prob = w.config0_rect(linear=linear)
    ref = oracle.rsrr(prob)
    h = open_nep(rs, prob)
    sample_rect(rs, prob, h)
    X = h.samples()
    assert rel_err_cols(X, ref["Shat"]).max() < 1e-8
    h.project(1e-14)
    lam, V, res = h.solve(500, 2, 1e3, 4096, True)
    info = h.info()
    h.close()
    assert info["n_winding"] == ref["n_winding"] == 14
    assert abs(complex(info["winding_re"], info["winding_im"]) - ref["winding"]) < 1e-7
    assert lam.size == ref["lam"].size == 14
    assert match(lam, ref["lam"]) < 1e-9
    assert scaled(prob, lam, res).max() < 1e-10
    if linear:
        h_ = 1.0 / 31
        l1 = 4 / h_ ** 2 * np.sin(np.arange(1, 31) * np.pi * h_ / 2) ** 2
        mu = (l1[:, None] + l1[None, :]).ravel()
        assert match(lam, mu[oracle.inside_contour(mu, prob.gamma, prob.a, prob.b, "rectangle")]) < 1e-9


def test_rectangle_moments_and_argument_checks(rs):
    """The moment scheme with the rectangle's Gauss-Legendre weights against the oracle, and
    the argument checks of rectangular contours."""
    prob = w.config0_rect(N=36, side_nodes=12)
    h = open_nep(rs, prob)
    sample_rect(rs, prob, h, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10)
    Shat = h.samples()
    kS = h.project_moments(18)
    S, P = h.basis(), h.projected()
    lam, V, res = h.solve(500, 2, 1e3, 4096, True)
    M = oracle.moment_matrix(prob, Shat, 18)
    ref_S, ref_sig, ref_k = oracle.truncated_basis(M, 1e-14)
    assert abs(kS - ref_k) <= near_threshold(ref_sig, 1e-14)
    assert np.linalg.norm(M - S @ (S.conj().T @ M), 2) <= 20 * 1e-14 * ref_sig[0] + 1e-15 * np.linalg.norm(M)
    ref = oracle.rsrr(prob, moments=18)
    assert lam.size == ref["lam"].size == 14
    assert match(lam, ref["lam"]) < 1e-9
    for kw in (dict(N=31), dict(side_nodes=18), dict(side_nodes=-1)):
        N = kw.get("N", prob.N)
        with pytest.raises(rs.RsrrError) as e:
            h.sample(prob.gamma, prob.a, prob.b, N, prob.L, prob.U[:, :prob.L], rs.RSRR_FP64, 1e-12, 12,
                     shape=rs.RSRR_CONTOUR_RECTANGLE, side_nodes=kw.get("side_nodes", 0))
        assert e.value.name == "EINVAL"
    with pytest.raises(rs.RsrrError) as e:
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12, shape=7)
    assert e.value.name == "EINVAL"
    sample_rect(rs, prob, h)
    h.project(1e-14)
    with pytest.raises(rs.RsrrError) as e:
        h.solve(501, 2, 1e3, 4096, True)
    assert e.value.name == "EINVAL"
    h.close()


@pytest.mark.parametrize("name,d", [("tiny_qep", 2), ("config0_flat", 20)])
def test_chebyshev_projection_matches_oracle(rs, name, d):
    """rsrr_project_chebyshev (Section 6.2, Eqs. eq-Ts-interp, eq-Ts-coefs): the d + 1
    interpolant coefficients P_hat_j against the oracle's on the device's basis, and the
    eigenvalues against the oracle's Chebyshev route, the direct route and (quadratic NEP) the
    companion linearisation; residuals are those of the true T."""
    if name == "config0_flat":
        prob = w.config0()
        prob.b = 10.0
        lo, hi, K = 100.0, 400.0, 2
    else:
        prob = w.by_name(name)
        lo, hi, K = prob.gamma.real - prob.a, prob.gamma.real + prob.a, 4
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
    kS = h.project_chebyshev(d, lo, hi)
    assert h.info()["red_terms"] == d + 1
    S, Ph = h.basis(), h.projected()
    lam, V, res = h.solve(500, K, 1e3, 4096, True)
    h.close()
    ref_Ph, _ = oracle.chebyshev_reduce(prob, S, d, lo, hi)
    assert np.abs(Ph - ref_Ph).max() < 1e-11 * np.abs(ref_Ph).max()
    ref = oracle.rsrr(prob, K=K, chebyshev=(d, lo, hi))
    assert lam.size == ref["lam"].size > 0
    assert match(lam, ref["lam"]) < 1e-9
    assert scaled(prob, lam, res).max() < 1e-10
    direct = oracle.rsrr(prob, K=K)
    assert match(lam, direct["lam"]) < 1e-9
    if name == "tiny_qep":
        assert match(lam, exact_eigs(name, prob)) < 1e-9


def test_chebyshev_argument_checks(rs):
    prob = w.tiny_qep()
    h = open_nep(rs, prob)
    with pytest.raises(rs.RsrrError) as e:
        h.project_chebyshev(4, -1.0, 1.0)
    assert e.value.name == "EORDER"
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
    for d, lo, hi in ((-1, -1.0, 1.0), (257, -1.0, 1.0), (4, 1.0, 1.0), (4, 2.0, -1.0)):
        with pytest.raises(rs.RsrrError) as e:
            h.project_chebyshev(d, lo, hi)
        assert e.value.name == "EINVAL"
    # a Chebyshev term can also be one of T's own functions
    fns = [(w.FN_CHEBYSHEV, [2, -1.6, 1.6]) if f.kind == w.FN_Z2 else (f.kind, f.params()) for f in prob.fns]
    h.close()
    h2 = rs.Nep(prob.n, prob.rowptr, prob.colind, prob.vals, fns)
    h2.close()


def tz_handle(rs, prob, tz):
    return rs.Nep.from_tz(prob.n, prob.rowptr, prob.colind, tz)


def test_tz_handle_equals_affine_handle(rs):
    """rsrr_create_nep_tz with T(z) = sum_i f_i(z) A_i supplied as values: the samples equal the
    affine handle's, and rsrr_project_chebyshev gives the affine handle's Chebyshev eigenvalues."""
    p = w.config0()
    p.b = 10.0
    F = lambda z: oracle.coefficients(p.fns, np.array([z]))[0][0]
    ha = open_nep(rs, p)
    hb = tz_handle(rs, p, lambda z: F(z) @ p.vals)
    out = []
    for h in (ha, hb):
        h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, rs.RSRR_FP64, 1e-12, 12)
        X = h.samples()
        h.project_chebyshev(16, 100.0, 400.0)
        lam, V, res = h.solve(500, 2, 1e3, 4096, True)
        out.append((X, lam, res))
        h.close()
    assert rel_err_cols(out[1][0], out[0][0]).max() < 1e-12
    assert out[1][1].size == out[0][1].size == 22
    assert match(out[1][1], out[0][1]) < 1e-11
    for X, lam, res in out:
        assert scaled(p, lam, res).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_distributed_delay_tz_matches_oracle(rs, prec):
    """A NEP known only by its values (one delay per coupling, Section 6's situation): samples,
    Chebyshev coefficients and eigenvalues against the oracle; residuals of the true T scaled
    by ||T(lambda)||_F; the tz handle refuses the term-by-term projections."""
    p = w.distributed_delay()
    lo, hi = p.gamma.real - p.a, p.gamma.real + p.a
    h = tz_handle(rs, p, p.tz)
    mode = rs.RSRR_FP64 if prec == "fp64" else rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL
    h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, mode, 1e-12 if prec == "fp64" else 1e-10, 20)
    X = h.samples()
    ref_X, infos, _ = oracle.sample(p)
    assert rel_err_cols(X, ref_X).max() < 1e-8
    for call in (lambda: h.project(1e-14), lambda: h.project_moments(8)):
        with pytest.raises(rs.RsrrError) as e:
            call()
        assert e.value.name == "EINVAL"
    with pytest.raises(rs.RsrrError) as e:
        h.solve(500, 2, 1e3, 4096, True)
    assert e.value.name == "EORDER"
    h.project_chebyshev(16, lo, hi)
    S, Ph = h.basis(), h.projected()
    ref_Ph, _ = oracle.chebyshev_reduce(p, S, 16, lo, hi)
    assert np.abs(Ph - ref_Ph).max() < 1e-11 * np.abs(ref_Ph).max()
    lam, V, res = h.solve(500, 2, 1e3, 4096, True)
    h.close()
    ref = oracle.rsrr(p, chebyshev=(16, lo, hi))
    assert lam.size == ref["lam"].size == 28
    assert match(lam, ref["lam"]) < 1e-9
    for t in range(lam.size):
        assert res[t] / np.linalg.norm(p.tz(lam[t])) < 1e-10
