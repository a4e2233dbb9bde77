"""Admission logic of the RSRR server (host only): arrival order, bypass by smaller requests
within the budget, the bypass limit that prevents starvation, and what happens to a request the
device refused for lack of memory (held until another request completes, bounded retries)."""
from types import SimpleNamespace

from paper_1510_07522_gb300.serve import after_enomem, footprint_bytes, select_admissible


def req(fp, bypassed=0, held_until=-1):
    return SimpleNamespace(footprint=fp, bypassed=bypassed, held_until=held_until, retries=0)


def test_oldest_fitting_request_first():
    q = [req(10), req(5), req(1)]
    assert select_admissible(q, 100, 4) == 0


def test_smaller_request_passes_a_blocked_one():
    q = [req(80), req(10), req(5)]
    i = select_admissible(q, 50, 4)
    assert i == 1 and q[0].bypassed == 1 and q[1].bypassed == 0


def test_bypass_limit_blocks_queue():
    q = [req(80, bypassed=4), req(10)]
    assert select_admissible(q, 50, 4) is None


def test_nothing_fits():
    assert select_admissible([req(80), req(90)], 50, 4) is None
    assert select_admissible([], 50, 4) is None


def test_footprint_is_persistent_plus_largest_phase():
    """S_hat and the CSR values stay; the sampling factors, the projection work and the reduced
    solve's inverses come one after another, so the bound is their maximum on top."""
    n, kl, ku, N, L, nnz, J = 40000, 200, 200, 64, 32, 200000, 3
    s_hat = n * N * L * 16
    persistent = s_hat + J * nnz * 16 + (64 << 20)
    # ten reduced points: the 64 band factors (~17 GB of complex64) are the largest phase
    a = footprint_bytes(n, kl, ku, N, L, nnz, J, N_S=10)
    b = footprint_bytes(n, kl, ku, 32, L, nnz, J, N_S=10)
    c = footprint_bytes(n, 100, 100, N, L, nnz, J, N_S=10)
    assert a > b and a > c
    assert 15e9 < a - persistent < 25e9
    # FP64 factors take twice the bytes
    assert footprint_bytes(n, kl, ku, N, L, nnz, J, False, N_S=10) - persistent > 1.9 * (a - persistent)
    # 500 reduced points of k_S <= N L = 2048 hit the 24 GiB cap and become the largest phase
    d = footprint_bytes(n, kl, ku, N, L, nnz, J)
    assert 24 * 2 ** 30 < d - persistent < 28e9


def test_enomem_alone_finishes_with_error():
    r = req(10)
    assert after_enomem(r, others_inflight=0, completions=5, max_retries=3) is False


def test_enomem_requeued_only_after_a_completion():
    r = req(10)
    assert after_enomem(r, others_inflight=2, completions=5, max_retries=3) is True
    q = [r, req(20)]
    assert select_admissible(q, 100, 4, completions=5) == 1     # held: skipped, not a bypass
    assert r.bypassed == 0
    assert select_admissible(q, 100, 4, completions=6) == 0     # one more request completed


def test_enomem_retries_are_bounded():
    r = req(10)
    outcomes = [after_enomem(r, others_inflight=1, completions=k, max_retries=3) for k in range(5)]
    assert outcomes == [True, True, True, False, False]
