"""The sampler autotuner (RSRR_AUTOTUNE): each handle's T(z_j) solves are timed on one sampling
point with the candidate strategies (band LU on tensor or CUDA cores, dense LU, band-part
preconditioned GMRES) and the fastest that meets the tolerance is used; choices are cached per
size bucket.  Whatever it picks, the samples must be those of the oracle's direct solves
(Algorithm 2, Step 2)."""
import numpy as np
import pytest

import oracle
import workloads as w
from gpu_util import fns_of, rel_err_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def tuned_handle(rs, p):
    return rs.Nep(p.n, p.rowptr, p.colind, p.vals, fns_of(p), rs.RSRR_NATURAL_ORDER | rs.RSRR_AUTOTUNE)


def test_time_delay_members_tuned_and_cached(rs):
    """Time-delay members (full band ~ n from the 5 % random coupling): the tuner compares the
    dense LU with GMRES on the grid Laplacian's band; the weight rule must find that band (the
    delay coupling is ~e^{-17} smaller), and a second member of the same size reuses the choice."""
    mode = rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL
    infos = []
    for idx in (0, 5):
        p = w.config3_member(idx, s=20, N=8, L=4)
        ref, _, _ = oracle.sample(p, dense=True)
        h = tuned_handle(rs, p)
        h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, mode, 1e-10, 40)
        info = h.info()
        infos.append(info)
        assert info["tune_strategy"] in (2, 3)
        if info["tune_strategy"] == 3:
            assert info["tune_band"] == 20 and info["iterative_band"] == 20
        assert h.eta().max() <= 1e-10
        assert rel_err_cols(h.samples(), ref).max() < 1e-8
        h.close()
    assert infos[0]["tune_cached"] == 0 and infos[1]["tune_cached"] == 1
    assert infos[1]["tune_strategy"] == infos[0]["tune_strategy"]


def test_banded_nep_tuned_to_a_band_lu(rs):
    """A grid NEP whose whole band is narrow: the direct band LU wins (no narrower band part holds
    the weight, so GMRES is not a candidate), and the samples are the oracle's."""
    p = w.config1(s=48, N=8, L=4)
    ref, _, _ = oracle.sample(p)
    h = tuned_handle(rs, p)
    h.sample(p.gamma, p.a, p.b, p.N, p.L, p.U, rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL, 1e-10, 20)
    info = h.info()
    assert info["tune_strategy"] in (0, 1) and info["iterative_band"] == -1
    assert rel_err_cols(h.samples(), ref).max() < 1e-9
    h.close()


def test_batch_with_autotune_equals_one_at_a_time(rs):
    probs = [w.config3_member(i, s=18, N=6, L=4) for i in (1, 2, 3)]
    mode = rs.RSRR_C64_IR | rs.RSRR_REFINE_FULL
    hs = [tuned_handle(rs, p) for p in probs]
    rs.sample_batch(hs, [(p.gamma, p.a, p.b) for p in probs], [p.N for p in probs], [p.L for p in probs],
                    [p.U for p in probs], mode, 1e-10, 40)
    for h, p in zip(hs, probs):
        ref, _, _ = oracle.sample(p, dense=True)
        assert h.info()["tune_strategy"] in (2, 3)
        assert rel_err_cols(h.samples(), ref).max() < 1e-8
        h.close()
