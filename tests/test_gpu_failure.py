"""Failure detection on the GPU without a fault: a bounded device wait that
nothing releases (a look-back scan tile whose predecessor never publishes)
gives up after its poll limit, records KPX_E_TIMEOUT in the planner's
status, and returns; the host reads the status, the planner stays stopped,
and the CUDA context stays usable for the next planner."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_02846_gb300 import scenes  # noqa: E402

KPX_E_TIMEOUT = 6


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


def test_bounded_wait_times_out_and_reports(kpx):
    prob = scenes.dubins_scene(0)
    pl = kpx.Planner(prob)
    pl.iterate(3)
    before = pl.header()
    assert before.status == kpx.KPX_OK
    t0 = time.perf_counter()
    assert kpx.load().kpx_debug_wait_timeout(pl.h) == kpx.KPX_OK
    waited = time.perf_counter() - t0
    h = pl.header()
    assert h.status == KPX_E_TIMEOUT
    assert h.err_info[0] == (0x10000 | 1)
    print("bounded wait gave up after %.3f s" % waited)
    assert waited < 10.0
    # the planner stays stopped: further iterations are no-ops
    pl.iterate(4)
    assert pl.header().iter == before.iter
    pl.close()
    # the context is still usable: a new planner plans as before
    a, b = kpx.Planner(prob), kpx.Planner(prob)
    a.iterate(5)
    b.iterate(5)
    sa, sb = a.arrays(), b.arrays()
    assert a.header().status == kpx.KPX_OK and a.header().iter == 5
    assert np.array_equal(sa["key"], sb["key"])
    a.close()
    b.close()
