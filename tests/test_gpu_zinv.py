"""The reduced solve's batched inverse (rsrr_zinv_batch: blocked Gauss-Jordan elimination with
partial pivoting, rank-b updates on the library's ZGEMM) against LAPACK's inverse on the host
(numpy.linalg.inv, a library routine standing in for the plain definition A X = I).

Bar: the inverse's normwise residual ||X A - I||_max / (||X||_max ||A||_max k) at FP64 rounding
level, and element-wise agreement with LAPACK within cond(A) times that level.  Sizes cover one
block, several blocks with a ragged last one (b = 32 up to k = 400, 16 beyond), k = 1, both
ZGEMM paths (FP64 CUDA cores, tensor-core emulation), pivoting that a zero diagonal forces, a
graded matrix, and a singular member of a batch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def run(rs, mats, path):
    import torch
    k = mats[0].shape[0]
    host = np.stack([m.T for m in mats])  # row-major storage of the transposes = column-major
    A = torch.from_numpy(np.ascontiguousarray(host)).to("cuda")
    info = torch.zeros(len(mats), dtype=torch.int32, device="cuda")
    rs.zinv_batch(path, A, info, k, len(mats))
    out = A.cpu().numpy()
    return [out[t].T for t in range(len(mats))], info.cpu().numpy()


def rand(rng, k):
    return rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))


def check(A, X, tol=2e-14):
    k = A.shape[0]
    R = X @ A - np.eye(k)
    assert np.abs(R).max() <= tol * k * np.abs(X).max() * np.abs(A).max()
    ref = np.linalg.inv(A)
    cond = np.linalg.cond(A)
    assert np.abs(X - ref).max() <= 1e-15 * k * cond * np.abs(ref).max()


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("k", [1, 5, 32, 33, 97, 403])
def test_inverse_matches_lapack(rs, path, k):
    rng = np.random.default_rng([k, path])
    mats = [rand(rng, k) for _ in range(3)]
    X, info = run(rs, mats, path)
    assert np.all(info == 0)
    for A, Xi in zip(mats, X):
        check(A, Xi)


def test_inverse_wide_block_16(rs):
    """k = 633 (the reduced size of the large benchmark problem): 16-column blocks."""
    rng = np.random.default_rng(633)
    mats = [rand(rng, 633) for _ in range(2)]
    X, info = run(rs, mats, 0)
    assert np.all(info == 0)
    for A, Xi in zip(mats, X):
        check(A, Xi)


def test_pivoting_and_grading(rs):
    """A zero diagonal (every elimination step must pivot) and rows graded over 8 decades."""
    rng = np.random.default_rng(7)
    k = 70
    A1 = rand(rng, k)
    np.fill_diagonal(A1, 0.0)
    A2 = np.diag(10.0 ** np.linspace(0, 8, k)) @ rand(rng, k)
    X, info = run(rs, [A1, A2], 2)
    assert np.all(info == 0)
    check(A1, X[0])
    check(A2, X[1])
    # the left residual of the graded matrix (cond 1.6e9), entry by entry: within 100 times
    # LAPACK's on the same matrix (Gauss-Jordan's bound is of the same form as LU's; an FP64 model
    # of this elimination gives 8 times LAPACK's, the emulated rank-b updates 4 times that)
    lapack = np.abs(np.linalg.inv(A2) @ A2 - np.eye(k)).max()
    assert np.abs(X[1] @ A2 - np.eye(k)).max() < 100 * lapack


def test_singular_member_is_flagged(rs):
    """A zero column in one member: info flags it, the other members are unaffected."""
    rng = np.random.default_rng(11)
    k = 45
    good = [rand(rng, k), rand(rng, k)]
    bad = rand(rng, k)
    bad[:, 17] = 0.0
    X, info = run(rs, [good[0], bad, good[1]], 0)
    assert list(info) == [0, 1, 0]
    check(good[0], X[0])
    check(good[1], X[2])
