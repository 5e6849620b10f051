"""GPU parity: every phase of the CUDA iteration against the FP64 oracle on
the same inputs, through the C ABI (ctypes binding).

Sizes: the DI and Dubins cases run every slot of an iteration (several warps,
tiles and a ragged tail); the full-size quadcopter and Dubins configurations
are checked on sampled slots that the oracle evaluates one by one, in the
same launch configuration the benchmark uses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2602_02846_gb300 import scenes  # noqa: E402

from tests import gpu_helpers as gh  # noqa: E402


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


def _run_lockstep(kpx, prob, iters, flags=0):
    pl = kpx.Planner(prob, flags=flags)
    reports = []
    for _ in range(iters):
        if pl.header().status != 0:
            break
        reports.append(gh.step_phases(pl, prob))
    return pl, reports


CASES = {
    "di_config": lambda: scenes.di_scene(0),
    "di_16grid": lambda: scenes.di_scene(1, grid_pos=16, tree_cap=32768),
    "di_adaptive": lambda: scenes.di_scene(2, grid_pos=15, tree_cap=100000, lam=0),
    "di_empty": lambda: scenes.di_scene(3, n_obstacles=0, grid_pos=12, tree_cap=20000),
    # one step count for every sample (k_min = k_max): equal sort keys, ties in slot order
    "di_fixed_k": lambda: scenes.di_scene(1, grid_pos=16, tree_cap=32768).replace(k_min=12, k_max=12),
    # a wide step-count range (1 to 300 steps): long rollouts, K spanning many values in each chunk
    "di_long_k": lambda: scenes.di_scene(1, grid_pos=16, tree_cap=32768).replace(k_min=1, k_max=300),
    "dubins_forest": lambda: scenes.dubins_scene(0),
    "dubins_open": lambda: scenes.dubins_scene(1, n_obstacles=0, tree_cap=1 << 16, lam=16),
    "quad_small": lambda: scenes.quad_scene(0, clutter=200, certify=False, tree_cap=1 << 16, lam=8),
    # anisotropic inertia: the general body-rate dynamics with the gyroscopic term
    "quad_aniso": lambda: _anisotropic(scenes.quad_scene(0, clutter=200, certify=False, tree_cap=1 << 16, lam=8)),
    # path-length cost: the quadcopter rollout loop's path-length variant
    "quad_pathlen": lambda: scenes.quad_scene(0, clutter=200, certify=False, tree_cap=1 << 16, lam=8).replace(
        cost_kind=scenes.COST_PATH_LENGTH, w_effort=0.0),
}


def _anisotropic(prob):
    p = list(prob.param)
    p[2:5] = [scenes.f32(0.008), scenes.f32(0.011), scenes.f32(0.015)]
    return prob.replace(param=p)


@pytest.mark.parametrize("case", list(CASES))
def test_iteration_lockstep(kpx, case):
    """Several consecutive iterations, each checked phase by phase."""
    prob = CASES[case]()
    iters = {"di_config": 6, "di_16grid": 6, "di_adaptive": 4, "di_empty": 5, "di_fixed_k": 5, "di_long_k": 4, "dubins_forest": 6,
             "dubins_open": 8, "quad_small": 3, "quad_aniso": 3, "quad_pathlen": 3}[case]
    pl, reps = _run_lockstep(kpx, prob, iters)
    assert reps, "no iteration ran"
    tot = sum(r["slots"] for r in reps)
    ex = sum(r["validity_exempt"] + r["region_exempt"] for r in reps)
    print(case, "slots", tot, "exempt", ex, "max err", max(r["max_state_err"] for r in reps),
          "nodes", reps[-1]["n_nodes"])
    assert ex <= max(2, 0.002 * tot)
    pl.close()


def test_capacity_rule_lockstep(kpx):
    """The iteration that overflows the tree is checked phase by phase; the
    planner then stays KPX_TREE_FULL and further iterations change nothing."""
    prob = scenes.di_scene(4, grid_pos=16, tree_cap=700)
    pl = kpx.Planner(prob)
    full_seen = False
    for _ in range(30):
        rep = gh.step_phases(pl, prob)
        if rep["full"]:
            full_seen = True
            break
    assert full_seen
    a = pl.arrays()
    assert a["n_nodes"] == 700
    st = pl.iterate(3, stats=True)
    assert st["status"] == kpx.KPX_TREE_FULL
    b = pl.arrays()
    assert b["iter"] == a["iter"]
    assert np.array_equal(a["region_key"], b["region_key"])
    pl.close()


def _sampled_propagate(kpx, prob, warm_iters, n_samples, seed=0):
    pl = kpx.Planner(prob)
    pl.iterate(warm_iters)
    before = pl.arrays()
    rec = pl.make_records()
    pl.debug_step("begin")
    pl.debug_step("propagate", rec)
    h = pl.header()
    ns = int(h.n_slots)
    rng = np.random.default_rng(seed)
    slots = np.unique(np.concatenate([rng.integers(0, ns, size=min(n_samples, ns)), [0, ns - 1]]))
    g = gh.records_host(rec, prob.n, prob.m, ns)
    tx, tc = gh.oracle_inputs(before)
    o = oracle.propagate(prob, int(h.iter), int(h.lam), tx, tc, before["VA"], int(h.count_A), slots=slots)
    rep = gh.compare_propagate(prob, g, o, slots=slots)
    rep["n_slots"] = ns
    pl.close()
    return rep


def test_quad_full_config_sampled(kpx):
    """12D quadcopter at its full configuration (2^22 nodes, 16^3 x 4^3
    regions, lambda 128, 1,000 boxes): sampled slots against the oracle."""
    prob = scenes.quad_scene(0)
    rep = _sampled_propagate(kpx, prob, warm_iters=4, n_samples=3000)
    print("quad", rep)
    assert rep["n_slots"] > 10000
    assert rep["validity_exempt"] + rep["region_exempt"] <= max(2, 0.002 * rep["slots"])


def test_quad_large_tree_lockstep(kpx):
    """The quadcopter at its full configuration (16^3 x 4^3 regions, lambda
    128, 2^22 capacity) among 1,000 boxes without the walls, grown past 10^6
    nodes; then one iteration phase by phase: sampled propagate slots, and in
    full the region argmin, the winners, the capacity rule, the appended rows,
    PruneNodes over every node (Alg. 3; the prune's look-back spans over a
    thousand tiles) and the next V_A."""
    prob = scenes.quad_scene(0, clutter=1000, certify=False, walls=False)
    pl = kpx.Planner(prob)
    pl.iterate(45)
    h = pl.header()
    assert h.n_nodes >= 1_000_000, h.n_nodes
    rep = gh.step_phases(pl, prob, sample_slots=4000)
    print("quad large tree", rep)
    assert rep["validity_exempt"] + rep["region_exempt"] <= max(2, 0.002 * rep["slots"])
    assert rep["n_nodes"] >= 1_000_000 and rep["winners"] > 1000
    pl.close()


def test_dubins_full_config_sampled(kpx):
    prob = scenes.dubins_scene(0)
    rep = _sampled_propagate(kpx, prob, warm_iters=10, n_samples=3000)
    print("dubins", rep)
    assert rep["validity_exempt"] + rep["region_exempt"] <= max(2, 0.002 * rep["slots"])


def _all_arrays(pl):
    """Every tree array and region key; not the header, nor region_snap (the
    capacity rule's scratch, unwritten until a snapshot is due)."""
    a = pl.arrays()
    return {k: v for k, v in a.items() if k not in ("header", "region_snap")}


def _same(a, b):
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8),
                                  np.ascontiguousarray(b[k]).view(np.uint8)), k
        else:
            assert a[k] == b[k], k


def test_production_iteration_equals_phases_and_early_reject(kpx):
    """kpx_iterate equals the phase-by-phase sequence bit for bit, and the
    early cost rejection (collision-after-cost) leaves every result unchanged."""
    prob = scenes.dubins_scene(2, n_obstacles=120, tree_cap=1 << 16, lam=32)
    pl = kpx.Planner(prob)
    pl.iterate(5)
    snap = pl.snapshot()
    pl.iterate(4)
    ref = _all_arrays(pl)
    pl.restore(snap)
    for _ in range(4):
        for ph in kpx.PHASES:
            pl.debug_step(ph)
    _same(ref, _all_arrays(pl))
    pl.close()
    pe = kpx.Planner(prob, flags=kpx.KPX_FLAG_EARLY_REJECT)
    pe.iterate(9)
    _same(ref, _all_arrays(pe))
    pe.close()


def _quad_order_keys(prob, x_nodes, va, lam, K, u, slots):
    """FP64 form of the quadcopter's order key: K, or the steps after which
    the velocity, extrapolated at the start's acceleration (thrust along the
    parent's body z axis, gravity), leaves its bounds."""
    node = va[slots // lam]
    xs = x_nodes[node].astype(np.float64)
    phi, th, psi = xs[:, 3], xs[:, 4], xs[:, 5]
    a = u[slots, 0].astype(np.float64) / float(prob.param[0])
    acc = [a * (np.cos(psi) * np.sin(th) * np.cos(phi) + np.sin(psi) * np.sin(phi)),
           a * (np.sin(psi) * np.sin(th) * np.cos(phi) - np.cos(psi) * np.sin(phi)),
           a * np.cos(th) * np.cos(phi) - float(prob.param[1])]
    n = K[slots].astype(np.float64)
    for i in range(3):
        v0 = xs[:, 6 + i]
        dv = acc[i] * float(prob.h)
        with np.errstate(divide="ignore", invalid="ignore"):
            up = np.where(dv > 0, (float(prob.x_hi[6 + i]) - v0) / dv, np.inf)
            down = np.where(dv < 0, (float(prob.x_lo[6 + i]) - v0) / dv, np.inf)
        n = np.minimum(n, np.minimum(up, down))
    return np.floor(np.maximum(n, 0.0))


@pytest.mark.parametrize("case", ["quad_full", "quad_small", "di_adaptive", "di_fixed_k", "dubins_forest"])
def test_slot_order_sorts_by_steps_and_leaves_results_unchanged(kpx, case):
    """The begin phase orders each 128-slot chunk by (key, offset), the key
    being K (the quadcopter's: K or its predicted step count): a permutation
    of the chunk whose live slots come first in non-decreasing key.  Rolling
    the slots out in that order changes no result: workspaces and the step,
    box-test and valid counters equal those of index order.  The
    quadcopter's key is checked against its FP64 form, to one step (the
    device rounds in FP32 with the hardware sine and cosine)."""
    prob = scenes.quad_scene(0) if case == "quad_full" else CASES[case]()
    iters = {"quad_full": 4, "quad_small": 4, "di_adaptive": 3, "di_fixed_k": 3, "dubins_forest": 8}[case]
    flags = kpx.KPX_FLAG_NO_FUSED
    pa = kpx.Planner(prob, flags=flags)
    pb = kpx.Planner(prob, flags=flags | kpx.KPX_FLAG_NO_SLOT_ORDER)
    pa.iterate(iters)
    pb.iterate(iters)
    # the order of the next iteration against the K the propagate records carry
    rec = pa.make_records()
    before = pa.arrays()
    pa.debug_step("begin")
    h = pa.header()
    ns = int(h.n_slots)
    order = pa.slot_order(ns)
    pa.debug_step("propagate", rec)
    pb.debug_step("begin")
    pb.debug_step("propagate")
    assert ns > 0 and order is not None and pb.slot_order(ns) is None
    K = rec["K"][:ns].cpu().numpy()
    quad = prob.m == 4
    if quad:
        u = rec["u"].view(prob.m, -1)[:, :ns].T.cpu().numpy()
    chunks = order.reshape(-1, 128).astype(np.int64)
    inversions = pairs = 0
    for c, perm in enumerate(chunks):
        assert np.array_equal(np.sort(perm), np.arange(128)), "chunk %d is not a permutation" % c
        live = min(128, ns - 128 * c)
        slots = 128 * c + perm[:live]
        assert np.all(slots < ns), "a dead slot sorted before a live one"
        if quad:
            qk = _quad_order_keys(prob, before["x"], before["VA"], int(h.lam), K, u, slots)
            assert np.all(np.diff(qk) >= -1), "chunk %d not in ascending predicted steps" % c
            inversions += int(np.sum(np.diff(qk) < 0))
            pairs += max(0, live - 1)
        else:
            key = K[slots].astype(np.int64) * 128 + perm[:live]
            assert np.all(np.diff(key) > 0), "chunk %d not in ascending (K, offset)" % c
    if quad:
        assert inversions <= 0.01 * pairs, (inversions, pairs)
    for ph in kpx.PHASES[2:]:
        pa.debug_step(ph)
        pb.debug_step(ph)
    pa.iterate(2)
    pb.iterate(2)
    _same(_all_arrays(pb), _all_arrays(pa))
    sa, sb = pa.iterate(0, stats=True), pb.iterate(0, stats=True)
    for k in ("total_valid", "total_steps", "total_box_tests", "total_candidates", "n_nodes"):
        assert sa[k] == sb[k], k
    pa.close()
    pb.close()


def test_determinism_and_reset(kpx):
    prob = scenes.di_scene(5, grid_pos=16, tree_cap=1 << 15)
    a = kpx.Planner(prob)
    b = kpx.Planner(prob)
    a.iterate(8)
    b.iterate(8)
    ra = _all_arrays(a)
    _same(ra, _all_arrays(b))
    b.iterate(3)
    b.reset()
    b.iterate(8)
    _same(ra, _all_arrays(b))
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["di_16grid", "dubins_open", "quad_small"])
def test_tree_invariants_fp64(kpx, case):
    """Every GPU tree edge re-rolled by the oracle in FP64 from the stored
    parent state: same end state (1e-4), valid, cost = parent + edge."""
    prob = CASES[case]()
    pl = kpx.Planner(prob)
    pl.iterate({"di_16grid": 5, "dubins_open": 12, "quad_small": 4}[case])
    a = pl.arrays()
    n = a["n_nodes"]
    assert n > 50
    cost = oracle.key_cost(a["key"]).astype(np.float64)
    worst = 0.0
    for i in range(1, min(n, 4000)):
        p = a["parent"][i]
        assert p < i
        r = oracle.rollout(prob, a["x"][p].astype(np.float64), a["u"][i], int(a["K"][i]))
        assert r["valid"] or r["margin"] < gh.NEAR
        worst = max(worst, float(gh.rel_err(a["x"][i], r["x_end"]).max()))
        assert abs(cost[i] - (cost[p] + r["edge_cost"])) <= gh.REL_TOL * max(1.0, cost[i])
    assert worst <= gh.REL_TOL
    # region keys: one node per visited region, V_A nodes are region-best
    rk = a["region_key"]
    visited = np.nonzero(rk != np.uint64(oracle.KEY_INF))[0]
    owners = {int(a["region"][i]) for i in range(n) if a["key"][i] == rk[a["region"][i]]}
    assert owners == set(int(r) for r in visited)
    act = np.nonzero(a["set"] == 1)[0]
    assert np.all(a["key"][act] == rk[a["region"][act]])
    pl.close()


def test_solution_revalidated_fp64(kpx):
    """The returned trajectory re-validates in FP64 segment by segment."""
    prob = scenes.di_scene(6, grid_pos=16, tree_cap=32768)
    pl = kpx.Planner(prob)
    st = pl.iterate(40, stats=True)
    tr = pl.best_trajectory()
    assert tr is not None, st
    rv = oracle.revalidate(prob, tr["states"].astype(np.float64), tr["controls"], tr["steps"])
    print("revalidate", rv, "cost", tr["cost"])
    assert rv["max_seg_err"] <= gh.REL_TOL
    assert rv["min_clearance"] >= -1e-4
    assert rv["goal_slack"] >= -1e-4
    assert abs(rv["cost"] - tr["cost"]) <= gh.REL_TOL * max(1.0, tr["cost"])
    assert np.allclose(tr["states"][0], prob.start)
    assert st["best_cost"] == np.float32(tr["cost"])
    pl.close()
