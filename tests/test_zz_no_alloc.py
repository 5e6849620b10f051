"""kpx_plan_static, the planning call that allocates nothing, gives the same
result as the allocating path.

Some callers cannot allocate device memory: real-time control loops that must
not wait on an allocator or fail mid-plan, and plugins whose host application
owns the device memory pool.  kpx_plan_static plans in the library's own
static device array instead.  Two calls in a row (on two different problems,
so the second call starts from the first call's leftovers in that shared
array) are compared with kpx_create + kpx_iterate + kpx_best_trajectory on a
caller workspace.  Both run the same phase kernels on the same inputs (the
workspace path's fused kernel is bit-identical to them), so the trajectories
must be equal bit for bit.

The call copies its result to the host and synchronises its stream, so it
cannot run while that stream is being captured into a CUDA graph: there it
must refuse with KPX_E_INVALID and leave the capture intact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2602_02846_gb300 import scenes  # noqa: E402


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
    assert np.array_equal(a["states"], b["states"])
    assert a["cost"] == b["cost"]


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


def test_static_plan_refuses_a_capturing_stream(kpx):
    prob = scenes.di_scene(7, grid_pos=16, tree_cap=32768)
    side = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        st, got = kpx.kpx_plan_static(prob, 5, stream=side)
        msg = kpx.last_create_error()
    assert st == kpx.KPX_E_INVALID and got is None
    assert "captured" in msg
    # the capture is intact: the graph replays the work recorded around the call
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    # and the call works again outside the capture
    st2, got2 = kpx.kpx_plan_static(prob, 30, stream=torch.cuda.current_stream())
    assert st2 == kpx.KPX_OK
    _same_trajectory(got2, _reference(kpx, prob, 30))


def kpx_static_limit():
    return 16 << 20
