"""Serving: requests that arrive while others run are admitted as slots and memory free up,
their work overlaps on the device, and each result equals the one computed alone."""
import numpy as np
import pytest

import workloads as w
from gpu_util import fns_of, match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def make_requests(rs, serve):
    probs = [w.config0(N=16, L=8, nx=12, ny=10), w.planted_sqrt(), w.tiny_qep(),
             w.config1b(s=16, N=24, L=8), w.planted_delay(), w.config0_linear(N=16, L=8, nx=14, ny=11),
             w.config3_member(2, s=12, N=16, L=8)]  # the last one takes the dense LU
    out = []
    for i, p in enumerate(probs):
        K = 4 if p.name == "tiny_qep" else 2
        out.append(serve.Request(rid=i, n=p.n, rowptr=p.rowptr, colind=p.colind, vals=p.vals, fns=fns_of(p),
                                 gamma=p.gamma, a=p.a, b=p.b, N=p.N, L=p.L, U=p.U, N_S=300, K=K))
    return out


def test_results_same_alone_and_in_mix(rs):
    from paper_1510_07522_gb300 import serve
    alone = {}
    srv = serve.Server(budget_bytes=64e9, slots=1)
    for r in make_requests(rs, serve):
        srv.submit(r)
        done = srv.wait(len(alone) + 1)
        alone[r.rid] = [d for d in done if d.rid == r.rid][0]
    srv.close()
    srv = serve.Server(budget_bytes=64e9, slots=4)
    mix = serve.replay(srv, make_requests(rs, serve), np.zeros(7))
    srv.close()
    assert srv.peak_inflight > 1  # requests really overlapped
    for r in mix:
        a = alone[r.rid]
        assert r.error is None and a.error is None, (r.error, a.error)
        assert r.lam.size == a.lam.size
        if r.lam.size:
            assert match(r.lam, a.lam) < 1e-9


def test_budget_limits_concurrency(rs):
    from paper_1510_07522_gb300 import serve
    reqs = make_requests(rs, serve)
    biggest = max(serve.footprint_bytes(r.n, *serve.band_of(r.n, r.rowptr, r.colind), r.N, r.L, r.colind.size,
                                        r.vals.shape[0]) for r in reqs)
    srv = serve.Server(budget_bytes=biggest, slots=4)
    done = serve.replay(srv, reqs, np.zeros(len(reqs)))
    srv.close()
    assert all(r.error is None for r in done)
    assert srv.in_use == 0


def test_request_larger_than_budget_is_refused(rs):
    from paper_1510_07522_gb300 import serve
    r = make_requests(rs, serve)[0]
    srv = serve.Server(budget_bytes=1e6, slots=1)
    srv.submit(r)
    done = srv.wait(1, timeout=30)
    srv.close()
    assert done[0].error and "budget" in done[0].error


def test_admission_footprint_bounds_measured_peak(rs):
    """The server admits a request when its estimated footprint fits the budget.  For each request
    type of the serving stream at its serving size (configs 0, 1, 2 and a time-delay member), the
    estimate must bound the device memory the request really holds at its peak (the library's
    pool high-water mark, measured with the request running alone)."""
    from paper_1510_07522_gb300 import serve
    import bench
    reqs = bench.serve_requests(serve, 4, 0, lambda t: (rs.RSRR_FP64 if t == "0" else rs.RSRR_C64_IR) | rs.RSRR_REFINE_FULL)
    by_type = {}
    for t in bench.SERVE_TYPES:   # one of each type, whatever the seeded draw gave
        p = bench.workload(t) if t != "3" else w.config3_member(7, s=40)
        prec = (rs.RSRR_FP64 if t == "0" else rs.RSRR_C64_IR) | rs.RSRR_REFINE_FULL
        by_type[t] = serve.Request(rid=int(t), n=p.n, rowptr=p.rowptr, colind=p.colind, vals=p.vals, fns=fns_of(p),
                                   gamma=p.gamma, a=p.a, b=p.b, N=p.N, L=p.L, U=p.U, precision=prec)
    assert len(reqs) == 4
    peaks = {}
    for t, r in by_type.items():
        kl, ku = serve.band_of(r.n, r.rowptr, r.colind)
        fp = serve.footprint_bytes(r.n, kl, ku, r.N, r.L, int(r.colind.size), int(r.vals.shape[0]),
                                   (r.precision & 0xff) == rs.RSRR_C64_IR)
        rs.lib().rsrr_device_peak_bytes(1)
        h = rs.Nep(r.n, r.rowptr, r.colind, r.vals, r.fns)
        h.sample(r.gamma, r.a, r.b, r.N, r.L, r.U, r.precision, r.tol, 20)
        h.project(r.delta)
        h.solve(r.N_S, r.K, 1e3, 4096, False)
        h.close()
        peaks[t] = (rs.lib().rsrr_device_peak_bytes(0), fp)
    for t, (peak, fp) in peaks.items():
        assert 0 < peak <= fp, (t, peaks)
