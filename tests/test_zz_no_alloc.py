"""kpx_plan_static, the planning call that allocates nothing, gives the same
result as the allocating path.

Some callers cannot allocate device memory: code recorded into a CUDA graph
(allocation is not allowed while a stream is captured), real-time control
loops that must not wait on an allocator or fail mid-plan, and plugins whose
host application owns the device memory pool.  kpx_plan_static plans in the
library's own static device array instead.  Two calls in a row (on two
different problems, so the second call starts from the first call's
leftovers in that shared array) are compared with kpx_create +
kpx_iterate + kpx_best_trajectory on a caller workspace, within the state
tolerance of the other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2602_02846_gb300 import scenes  # noqa: E402

REL_TOL = 1e-4


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


def _reference(kpx, prob, iters):
    pl = kpx.Planner(prob)
    pl.iterate(iters)
    tr = pl.best_trajectory()
    pl.close()
    return tr


def _same_trajectory(a, b):
    assert (a is None) == (b is None)
    if a is None:
        return
    assert a["steps"].shape == b["steps"].shape
    assert np.array_equal(a["steps"], b["steps"])
    assert np.array_equal(a["controls"], b["controls"])
    err = np.abs(a["states"].astype(np.float64) - b["states"]) / np.maximum(1.0, np.abs(b["states"]))
    assert err.max() <= REL_TOL
    assert abs(a["cost"] - b["cost"]) <= REL_TOL * max(1.0, abs(b["cost"]))


def test_static_plan_matches_workspace_path_twice(kpx):
    stream = torch.cuda.current_stream()
    problems = [
        (scenes.di_scene(7, grid_pos=16, tree_cap=32768), 30),
        (scenes.dubins_scene(1, n_obstacles=0, tree_cap=1 << 14, lam=16), 25),
    ]
    for prob, iters in problems:
        assert kpx.kpx_workspace_size(prob) <= kpx_static_limit()
        st, got = kpx.kpx_plan_static(prob, iters, stream=stream)
        ref = _reference(kpx, prob, iters)
        assert st in (kpx.KPX_OK, kpx.KPX_NO_SOLUTION)
        assert ref is not None, "test problem should reach the goal"
        _same_trajectory(got, ref)


def test_static_plan_rejects_oversized_problem(kpx):
    prob = scenes.dubins_scene(0)  # tree capacity 2^20: far above the static limit
    assert kpx.kpx_workspace_size(prob) > kpx_static_limit()
    st, got = kpx.kpx_plan_static(prob, 1, stream=torch.cuda.current_stream())
    assert st == kpx.KPX_E_NOMEM and got is None
    assert "static scratch" in kpx.last_create_error()


def kpx_static_limit():
    return 16 << 20
