"""The library's complex GEMM (rsrr_zgemm): the FP64 CUDA-core kernel and the FP64-accurate
tensor-core emulation (exact BF16 digit products, FP32 accumulation, FP64 combination) against
a plain complex128 reference of the same product on the host.

Bar: |C - C_ref|_ij <= 4 (K + 2) 2^-52 |alpha| max_k |op(A)_ik|_inf max_k |op(B)_kj|_inf
(|z|_inf = max(|Re z|, |Im z|)), the normwise size of an FP64 GEMM's rounding, plus 2^-52 of
|beta C|.  Shapes cover tile tails, both orientations of the tensor-core tiles, split K and
batches; rows and columns of widely different magnitudes and all-zero rows check the scaling."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def dev(X):
    """complex128 column-major device copy of the host matrix X (returns tensor, ld)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda")
    return t, X.shape[0]


def rand(rng, r, c, spread=0.0, zero_rows=()):
    X = (rng.normal(size=(r, c)) + 1j * rng.normal(size=(r, c))) * 10.0 ** rng.uniform(-spread, spread, (r, 1))
    X = X * 10.0 ** rng.uniform(-spread, spread, (1, c))
    for i in zero_rows:
        if i < r:
            X[i] = 0
    return X


def inf(X, axis):
    return np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=axis)


CASES = [  # M, N, K, opA, opB, spread
    (1, 1, 1, 0, 0, 0), (5, 7, 3, 0, 0, 0), (64, 32, 32, 0, 0, 0), (65, 33, 70, 2, 0, 0),
    (130, 45, 300, 0, 1, 3), (40, 200, 1000, 1, 2, 0), (300, 40, 5000, 2, 0, 2), (97, 96, 2049, 0, 0, 6),
]


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("M,N,K,oa,ob,spread", CASES)
def test_zgemm_matches_reference(rs, path, M, N, K, oa, ob, spread):
    import torch
    rng = np.random.default_rng([M, N, K, oa, ob])
    a = rand(rng, M, K, spread, zero_rows=(2,))
    b = rand(rng, K, N, spread)
    A = a if oa == 0 else a.T.copy() if oa == 1 else a.conj().T.copy()  # stored so that op(A) = a
    B = b if ob == 0 else b.T.copy() if ob == 1 else b.conj().T.copy()
    C0 = rand(rng, M, N)
    alpha, beta = 0.7 - 0.3j, -0.4 + 0.9j
    dA, lda = dev(A)
    dB, ldb = dev(B)
    dC, ldc = dev(C0)
    rs.zgemm(path, dA, dB, dC, oa, ob, alpha, beta, M=M, N=N, K=K, lds=(lda, ldb, ldc))
    torch.cuda.synchronize()
    C = dC.cpu().numpy().T
    ref = alpha * (a @ b) + beta * C0
    bound = 4 * (K + 2) * 2.0 ** -52 * abs(alpha) * np.outer(inf(a, 1), inf(b, 0)) + 2.0 ** -52 * np.abs(beta * C0)
    assert np.all(np.abs(C - ref) <= bound + 1e-300)


@pytest.mark.parametrize("path", [1, 2])
def test_zgemm_batched_with_shared_operand(rs, path):
    """batch of 3 with A shared (stride 0), B and C strided, beta = 0 (C's old values ignored)."""
    import torch
    rng = np.random.default_rng(11)
    M, N, K, nb = 70, 50, 600, 3
    a = rand(rng, M, K)
    bs = [rand(rng, K, N, 1) for _ in range(nb)]
    dA, lda = dev(a)
    dB = torch.from_numpy(np.ascontiguousarray(np.stack([x.T for x in bs]))).to("cuda")
    dC = torch.full((nb, N, M), complex("nan"), dtype=torch.complex128, device="cuda")
    rs.zgemm(path, dA, dB, dC, 0, 0, 1.0, 0.0, M=M, N=N, K=K, batch=nb, strides=(0, K * N, M * N),
             lds=(lda, K, M))
    torch.cuda.synchronize()
    for t in range(nb):
        C = dC[t].cpu().numpy().T
        ref = a @ bs[t]
        bound = 4 * (K + 2) * 2.0 ** -52 * np.outer(inf(a, 1), inf(bs[t], 0))
        assert np.all(np.abs(C - ref) <= bound)


def test_zgemm_argument_checks(rs):
    import torch
    x = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    for kw in (dict(path=3), dict(oa=5), dict(lds=(2, 4, 4))):
        with pytest.raises(rs.RsrrError) as e:
            rs.zgemm(kw.get("path", 2), x, x, x, kw.get("oa", 0), 0, 1.0, 0.0, M=4, N=4, K=4, lds=kw.get("lds", (4, 4, 4)))
        assert e.value.name == "EINVAL"


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1.0), (1.0, 0.0), (-1.0, 0.0), (2.5, 1.0), (1j, 1.0)])
def test_zgemm_update_forms_and_extreme_scales(rs, path, alpha, beta):
    """The forms the trailing updates use (alpha = -1, beta = 1 and the like), with rows and
    columns scaled from 1e-310 (subnormal inputs) to 1e300, so that results run from the
    subnormal range to 1e305: the digit and scale steps' slow paths and the fast ones agree."""
    import torch
    rng = np.random.default_rng([int(abs(alpha) * 10), int(abs(beta))])
    M, N, K = 70, 40, 96
    a = rand(rng, M, K)
    b = rand(rng, K, N)
    rs_ = np.ones(M)
    rs_[:4] = [1e300, 1e-300, 1e-310, 1e-200]
    cs_ = np.ones(N)
    cs_[:3] = [1e-5, 1e5, 1e-100]
    a = a * rs_[:, None]
    b = b * cs_[None, :]
    C0 = rand(rng, M, N) * rs_[:, None] * cs_[None, :]
    dA, lda = dev(a)
    dB, ldb = dev(b)
    dC, ldc = dev(C0)
    rs.zgemm(path, dA, dB, dC, 0, 0, alpha, beta, M=M, N=N, K=K, lds=(lda, ldb, ldc))
    torch.cuda.synchronize()
    C = dC.cpu().numpy().T
    ref = alpha * (a @ b) + beta * C0
    bound = 4 * (K + 2) * 2.0 ** -52 * abs(alpha) * np.outer(inf(a, 1), inf(b, 0)) + 2.0 ** -52 * np.abs(beta * C0)
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - ref) <= bound + K * 1e-320)
