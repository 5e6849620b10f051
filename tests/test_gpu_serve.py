"""The request loop on the GPU: every served query ends bit-identical to the
same problem planned alone (kpx_create + kpx_iterate for its budget), though
it was admitted into a recycled slot, in arena memory another query used
before, and iterated beside whatever else was resident.  Each served tree and
solution is also checked against the FP64 oracle directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_02846_gb300 import scenes  # noqa: E402
from paper_2602_02846_gb300.serve import Request, Server, summarize  # noqa: E402

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
    a.pop("region_snap")
    return a


def _same(a, b, label):
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8),
                                  np.ascontiguousarray(b[k]).view(np.uint8)), "%s: %s differs" % (label, k)
        else:
            assert a[k] == b[k], "%s: %s differs" % (label, k)


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        kind = int(rng.integers(3))
        s = int(rng.integers(1 << 20))
        if kind == 0:
            p = scenes.di_scene(s, grid_pos=16, n_obstacles=int(rng.integers(0, 60)),
                                tree_cap=int(rng.choice([4096, 16384, 32768])))
        elif kind == 1:
            p = scenes.dubins_scene(s, n_obstacles=int(rng.integers(0, 120)), tree_cap=1 << 15,
                                    lam=int(rng.choice([16, 32])))
        else:
            p = scenes.quad_scene(s, clutter=int(rng.integers(10, 150)), certify=False, tree_cap=1 << 15, lam=4)
        if r == 5:
            p = scenes.di_scene(s, grid_pos=16, tree_cap=700)    # fills its tree before its budget
        out.append(Request(r, p, 0.0, int(rng.integers(3, 17))))
    return out


def test_served_results_equal_planning_alone(kpx):
    reqs = _requests(30, seed=11)
    captured = {}

    def grab(req, out, member):
        captured[req.rid] = (_arrays(member), member.best_trajectory())

    # 3 slots per class and an arena that holds only a few trees at once:
    # queries wait, slots and memory are recycled, residents come and go
    sizes = sorted(kpx.kpx_workspace_size(r.problem) for r in reqs)
    srv = Server.create(memory_bytes=3 * sizes[-1], slots_per_class=3, iters_per_round=3, on_finish=grab)
    out = srv.serve(reqs, realtime=False)
    assert srv.arena.in_use == 0
    reused = len({o.slot for o in out}) < len(out)
    assert reused
    n_solved = 0
    for r, o in zip(reqs, out):
        assert o.status in ("done", "tree_full"), (r.rid, o.status)
        single = kpx.Planner(r.problem)
        single.iterate(r.iter_budget)
        ref = _arrays(single)
        got, traj = captured[r.rid]
        _same(ref, got, "request %d" % r.rid)
        ts = single.best_trajectory()
        assert (ts is None) == (traj is None)
        if ts is not None:
            assert np.array_equal(ts["states"], traj["states"]) and ts["cost"] == traj["cost"]
            assert o.cost == ts["cost"]
        assert o.iterations == int(ref["counters"][1])
        single.close()
        # the served tree and solution against the FP64 oracle (no CUDA planner in between)
        rep = gh.check_tree_fp64(r.problem, got, max_nodes=1500)
        assert rep["validity_exempt"] <= max(2, 0.002 * rep["checked"]), (r.rid, rep)
        if traj is not None:
            gh.revalidate_trajectory(r.problem, traj)
            n_solved += 1
    assert n_solved >= 1
    assert out[5].status == "tree_full" and out[5].n_nodes == 700
    srv.batch.close()


def test_realtime_stream_summary(kpx):
    reqs = [Request(i, p, t, 8) for i, (t, p) in enumerate(scenes.poisson_requests(100.0, 0.3, seed=4))]
    srv = Server.create(memory_bytes=4 << 30, slots_per_class=8, iters_per_round=4)
    import time
    t0 = time.perf_counter()
    out = srv.serve(reqs)
    wall = time.perf_counter() - t0
    s = summarize(out, srv.offset, wall)
    assert s["served"] == len(reqs) and s["rejected"] == 0
    for o in out:
        assert o.admitted >= o.arrival and o.finished > o.admitted
        if o.t_first is not None:
            # the first solution is seen after admission and before the harvest
            assert o.admitted - 1e-3 <= o.t_first <= o.finished + 1e-3
    srv.batch.close()
