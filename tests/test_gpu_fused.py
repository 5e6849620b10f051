"""The fused iteration (whole iterations in one cluster launch while the
problem is small) against the phase kernels: kpx_iterate with and without
KPX_FLAG_NO_FUSED ends bit-identical.  The cases cover problems that stay
small, problems that outgrow the fused kernel in the middle of a graph launch
(the phase kernels take over the remaining iterations through the
conditional node), the capacity rule inside the fused kernel, the early cost
rejection, and calls of different sizes (each kpx_iterate call is one launch
of the planner's graph, whose count node changes with the size)."""
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


def _state(pl, work_counts=True):
    """Arrays and counters.  work_counts=False leaves out the valid, step and
    box-test counts: with the early cost rejection they depend on the order in
    which slots reach the region-key check (a slot checked after a better
    valid key landed skips its obstacle pass), while every result does not."""
    a = pl.arrays()
    h = a.pop("header")
    a["counters"] = np.array([h.status, h.iter, h.n_nodes, h.count_A, h.first_solution_iter, h.n_active,
                              h.n_inactive, h.n_terminal, h.lam], np.int64)
    if work_counts:
        a["totals"] = np.array([h.total_candidates, h.total_valid, h.total_winners, h.total_steps,
                                h.total_box_tests, h.goal_key, h.last_candidates, h.last_valid, h.last_winners],
                               np.uint64)
    else:
        a["totals"] = np.array([h.total_candidates, h.total_winners, h.goal_key, h.last_candidates,
                                h.last_winners], np.uint64)
    a.pop("region_snap")  # scratch of the capacity rule: unwritten until a snapshot is due
    return a


def _same(a, b, label):
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8),
                                  np.ascontiguousarray(b[k]).view(np.uint8)), "%s: %s differs" % (label, k)
        else:
            assert a[k] == b[k], "%s: %s differs" % (label, k)


CASES = {
    # stays small for the whole run (the confined forest airplane)
    "dubins_forest": (lambda: scenes.dubins_scene(0), 37, 0),
    # the literal double-integrator configuration (stalls at a few dozen nodes)
    "di_literal": (lambda: scenes.di_scene(0), 40, 0),
    # grows past one chunk per warp within a few iterations: the switch to
    # the phase kernels happens inside a graph launch
    "dubins_open_growing": (lambda: scenes.dubins_scene(3, n_obstacles=0, tree_cap=1 << 16, lam=16), 29, 0),
    "di16_growing": (lambda: scenes.di_scene(1, grid_pos=16, tree_cap=32768), 35, 0),
    # the tree fills inside the fused kernel: capacity rule + snapshot
    "di_capacity": (lambda: scenes.di_scene(4, grid_pos=16, tree_cap=700), 33, 0),
    "quad_small": (lambda: scenes.quad_scene(1, clutter=100, certify=False, tree_cap=1 << 15, lam=4), 21, 0),
    "dubins_early_reject": (lambda: scenes.dubins_scene(2, n_obstacles=120, tree_cap=1 << 16, lam=32), 19, 1),
    # outgrows the fused kernel after a few iterations, then fills its tree
    # inside the loop of phase kernels: the loop drops the iterations left
    "quad_fills_in_loop": (lambda: scenes.quad_scene(0, clutter=120, certify=False, walls=False, tree_cap=1 << 16,
                                                     lam=32), 40, 0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fused_equals_phase_kernels(kpx, case):
    make, iters, early = CASES[case]
    prob = make()
    flags = kpx.KPX_FLAG_EARLY_REJECT if early else 0
    fused = kpx.Planner(prob, flags=flags)
    plain = kpx.Planner(prob, flags=flags | kpx.KPX_FLAG_NO_FUSED)
    # uneven call sizes, and calls that start in the middle of the
    # problem's growth
    done = 0
    for n in (3, 16, iters - 19):
        fused.iterate(n)
        plain.iterate(n)
        done += n
        _same(_state(plain, not early), _state(fused, not early), "%s after %d iterations" % (case, done))
    if case in ("di_capacity", "quad_fills_in_loop"):
        assert fused.header().status == kpx.KPX_TREE_FULL
    if case == "quad_fills_in_loop":
        h = fused.header()
        assert 0 < h.fused_iterations < h.iter < 40 and h.graph_pending == 0
    tf, tp = fused.best_trajectory(), plain.best_trajectory()
    assert (tf is None) == (tp is None)
    if tf is not None:
        assert np.array_equal(tf["states"], tp["states"]) and tf["cost"] == tp["cost"]
    fused.close()
    plain.close()


def test_one_launch_per_call_and_count_updates(kpx):
    """kpx_iterate(n) is one graph launch that runs exactly n iterations,
    whatever the previous call's n was (the graph's count node changes only
    when n does)."""
    prob = scenes.dubins_scene(0)
    pl = kpx.Planner(prob)
    mx, fused = pl.graph_info()
    assert fused and mx > 1000
    assert kpx.Planner.launch_plan(200, mx) == [200]
    done, t_prev = 0, 0
    for n in (5, 5, 1, 37, 37, 2, 16):
        pl.iterate(n)
        done += n
        h = pl.header()
        assert h.iter == done and h.fused_iterations == done and h.graph_pending == 0
        # device clock: the launch's first iteration began after the
        # planner's start, and its last one ended after it began
        assert 0 < h.t_start_ns < h.t_last_ns
        assert h.first_solution_iter < 0 or h.t_start_ns <= h.t_first_solution_ns <= h.t_last_ns
        assert h.t_last_ns > t_prev
        t_prev = h.t_last_ns
    pl.close()


def test_fused_reset_and_restore(kpx):
    prob = scenes.di_scene(1, grid_pos=16, tree_cap=32768)
    pl = kpx.Planner(prob)
    pl.iterate(20)
    ref = _state(pl)
    snap = pl.snapshot()
    pl.iterate(7)
    pl.restore(snap)
    _same(ref, _state(pl), "restore")
    pl.reset()
    pl.iterate(20)
    _same(ref, _state(pl), "reset")
    pl.close()
