"""Failure detection on the device without a fault: every wait in the
library's kernels is bounded.  The self-test kernel waits on an mbarrier that
can never complete (it expects two arrivals and gets one); the wait gives up
after its fixed number of polls, the status word reports the timeout, the
call returns PIC_ERR_TIMEOUT, and the CUDA context stays usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def picrr():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1008_1685_gb300 as m

    return m


def test_bounded_wait_reports_timeout_and_context_survives(picrr):
    rc, sec = picrr.selftest_wait_timeout(0)
    assert rc == -5  # PIC_ERR_TIMEOUT
    assert sec < 30.0
    g = picrr.Sim(length_lambda=4, cells_per_lambda=100, seed=2)
    g.load_foil(1.0, 0.5, 20.0, 1, 1.0, 16)
    g.inject_laser(60.0, picrr.LP, picrr.ENV_SIN2, 3.0)
    assert g.step(100) == 100
    assert np.all(np.isfinite(g.field(picrr.EY)))
    g.close()
