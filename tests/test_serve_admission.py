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


def test_footprint_grows_with_band_and_points():
    a = footprint_bytes(40000, 200, 200, 64, 32, 200000, 3)
    b = footprint_bytes(40000, 200, 200, 32, 32, 200000, 3)
    c = footprint_bytes(40000, 100, 100, 64, 32, 200000, 3)
    assert a > b and a > c
    # 64 points of a band-200 problem: ~17.5 GB of factors, S_hat and the projection work, and
    # the reduced solve's inverses (k_S <= N L = 2048: capped at 24 GiB)
    assert 15e9 < a < 80e9
    d = footprint_bytes(40000, 200, 200, 64, 32, 200000, 3, N_S=50)
    # 500 points of k_S = 2048 hit the cap (25.8 GB), 50 points take 50 x 0.34 GB
    assert 7e9 < a - d < 10e9


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
