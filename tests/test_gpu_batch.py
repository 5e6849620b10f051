"""Batched planning (kpx_batch_*): every problem of a mixed batch ends
bit-identical to the same problem planned alone with kpx_create, whatever
else is in the batch (the problems share launches, not state), and every
member's tree and solution are checked against the FP64 oracle directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_02846_gb300 import scenes  # noqa: E402

from tests import gpu_helpers as gh  # noqa: E402


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


def _arrays(pl):
    a = pl.arrays()
    h = a.pop("header")
    a["counters"] = np.array([h.status, h.iter, h.n_nodes, h.count_A, h.first_solution_iter, h.n_active,
                              h.n_inactive, h.n_terminal], np.int64)
    a["totals"] = np.array([h.total_candidates, h.total_valid, h.total_winners, h.total_steps,
                            h.total_box_tests], np.uint64)
    a.pop("region_snap")  # only meaningful when the capacity rule is possible
    return a


def _same(a, b, label):
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8),
                                  np.ascontiguousarray(b[k]).view(np.uint8)), "%s: %s differs" % (label, k)
        else:
            assert a[k] == b[k], "%s: %s differs" % (label, k)


def _mixed_problems():
    return [
        scenes.dubins_scene(0, tree_cap=1 << 16),
        scenes.di_scene(1, grid_pos=16, tree_cap=32768),
        scenes.quad_scene(0, clutter=200, certify=False, tree_cap=1 << 16, lam=8),
        scenes.di_scene(0),
        scenes.dubins_scene(1, n_obstacles=0, tree_cap=1 << 14, lam=16),
        scenes.di_scene(2, grid_pos=15, tree_cap=20000, lam=0),
        scenes.di_scene(4, grid_pos=16, tree_cap=700),          # overflows: KPX_TREE_FULL mid-run
        scenes.quad_scene(1, clutter=100, certify=False, tree_cap=1 << 15, lam=4),
    ]


def test_batch_members_equal_single_planners(kpx):
    probs = _mixed_problems()
    iters = 12
    batch = kpx.BatchPlanner(probs)
    batch.iterate(iters)
    for i, prob in enumerate(probs):
        single = kpx.Planner(prob)
        single.iterate(iters)
        _same(_arrays(single), _arrays(batch.member(i)), "problem %d" % i)
        ts, tb = single.best_trajectory(), batch.member(i).best_trajectory()
        assert (ts is None) == (tb is None)
        if ts is not None:
            assert np.array_equal(ts["states"], tb["states"]) and ts["cost"] == tb["cost"]
        single.close()
    st = batch.member(6).iterate(0, stats=True)
    assert st["status"] == kpx.KPX_TREE_FULL and st["n_nodes"] == 700
    # reset puts every problem back to its create state
    batch.reset()
    batch.iterate(3)
    single = kpx.Planner(probs[1])
    single.iterate(3)
    _same(_arrays(single), _arrays(batch.member(1)), "after reset")
    batch.close()


def test_large_mixed_batch_sampled(kpx):
    rng = np.random.default_rng(7)
    probs = []
    for k in range(64):
        kind = k % 3
        if kind == 0:
            probs.append(scenes.di_scene(int(rng.integers(1000)), grid_pos=int(rng.integers(8, 17)),
                                         tree_cap=int(rng.choice([4096, 16384, 32768]))))
        elif kind == 1:
            probs.append(scenes.dubins_scene(int(rng.integers(1000)), n_obstacles=int(rng.integers(0, 120)),
                                             tree_cap=1 << 15, lam=int(rng.choice([16, 32]))))
        else:
            probs.append(scenes.quad_scene(int(rng.integers(1000)), clutter=int(rng.integers(10, 200)),
                                           certify=False, tree_cap=1 << 15, lam=4))
    iters = 8
    batch = kpx.BatchPlanner(probs)
    batch.iterate(iters)
    for i in range(0, 64, 7):
        single = kpx.Planner(probs[i])
        single.iterate(iters)
        _same(_arrays(single), _arrays(batch.member(i)), "problem %d" % i)
        single.close()
    batch.close()


def _results(pl):
    """Everything but the box-test counter (a work count that the obstacle
    grid's cell size changes by design)."""
    a = _arrays(pl)
    a["totals"] = a["totals"][:4]
    return a


def test_launch_settings_leave_results_unchanged(kpx):
    """Propagate grid size and obstacle-grid cell size, set before or during
    a run, change no result."""
    prob = scenes.quad_scene(1, clutter=100, certify=False, tree_cap=1 << 15, lam=4)
    ref = kpx.Planner(prob, flags=kpx.KPX_FLAG_NO_FUSED)
    ref.iterate(10)
    want = _results(ref)
    tests_ref = ref.header().total_box_tests
    ref.close()
    moved = False
    for bps, scale in [(1, 0.5), (2, 2.0), (0, 4.0)]:
        pl = kpx.Planner(prob, flags=kpx.KPX_FLAG_NO_FUSED)
        pl.set_launch(bps, scale)
        pl.iterate(4)
        pl.set_launch(0, 1.0)
        pl.iterate(6)
        _same(want, _results(pl), "blocks %d scale %g" % (bps, scale))
        moved |= pl.header().total_box_tests != tests_ref
        pl.close()
    assert moved  # the grid scale does change the work


def test_autotune_keeps_results(kpx):
    probs = _mixed_problems()
    ref = kpx.BatchPlanner(probs)
    ref.iterate(7)
    tuned = kpx.BatchPlanner(probs)
    tuned.iterate(3)
    report = tuned.autotune(iters=2, blocks=(0, 2), scales=(0.5, 2.0))
    assert set(report) == {(int(p.dyn), int(p.integ)) for p in probs}
    tuned.iterate(4)
    for i in range(len(probs)):
        _same(_results(ref.member(i)), _results(tuned.member(i)), "problem %d" % i)
    ref.close()
    tuned.close()


def test_batch_members_match_the_oracle(kpx):
    """Every member of a mixed batch (the three systems, adaptive lambda and a
    problem that overflows its tree among them) against the FP64 oracle, with
    no single-problem planner in between: each tree edge re-rolled in FP64,
    regions, keys, region ownership, node sets and the solution key, and each
    node's control and step count as the Philox draw of its parent at the
    iteration that appended it, in slot order (Alg. 2-4 per problem); every
    returned trajectory re-validated by the oracle."""
    probs = _mixed_problems()
    iters = 10
    batch = kpx.BatchPlanner(probs)
    B = len(probs)
    sizes = [[1] for _ in range(B)]
    lams = [[] for _ in range(B)]
    for _ in range(iters):
        batch.iterate(1)
        for i in range(B):
            h = batch.member(i).header()
            sizes[i].append(int(h.n_nodes))
            lams[i].append(int(h.lam))
    solved = 0
    for i, prob in enumerate(probs):
        a = batch.member(i).arrays()
        n = int(a["n_nodes"])
        created = np.searchsorted(np.asarray(sizes[i]), np.arange(n), side="right") - 1
        rep = gh.check_tree_fp64(prob, a, created=created, lam_at=lams[i], max_nodes=3000)
        print("member", i, prob.name, rep)
        assert rep["validity_exempt"] <= max(2, 0.002 * rep["checked"])
        tr = batch.member(i).best_trajectory()
        if tr is not None:
            gh.revalidate_trajectory(prob, tr)
            solved += 1
    full = batch.member(6).iterate(0, stats=True)
    assert full["status"] == kpx.KPX_TREE_FULL and full["n_nodes"] == 700
    assert solved >= 2
    batch.close()
