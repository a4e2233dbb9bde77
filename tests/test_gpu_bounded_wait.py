"""Every device-side wait of the library is bounded: a wait that cannot complete gives up after
its poll limit, the kernel returns, the call reports RSRR_ETIMEOUT, and the device stays usable.
The waits are made to run out from the host (a grid-barrier arrival count no CTA can complete,
an mbarrier phase nothing arrives at), never by faulting the device."""
import numpy as np
import pytest

import workloads as w
from gpu_util import open_nep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_that_cannot_complete_reports_timeout(rs, kind):
    with pytest.raises(rs.RsrrError) as e:
        rs.rsrr_selftest_bounded_wait(kind)
    assert e.value.name == "ETIMEOUT"


@pytest.mark.parametrize("kind", [2, 3])
def test_same_wait_completes_when_satisfiable(rs, kind):
    rs.rsrr_selftest_bounded_wait(kind)


def test_device_usable_after_timeouts(rs):
    for kind in (0, 1, 0):
        with pytest.raises(rs.RsrrError):
            rs.rsrr_selftest_bounded_wait(kind)
    prob = w.config0(N=4, L=2, nx=8, ny=8)
    h = open_nep(rs, prob)
    h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12)
    assert h.eta().max() <= 1e-13
    h.close()
