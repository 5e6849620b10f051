"""Oracle pins at the level of the whole loop (Alg. 1): tree invariants after
every iteration, cost lower bounds, monotone solution cost, the capacity
rule, and FP64 re-validation of the returned trajectory.

Invariants (from Assumption 1 and Alg. 2-4): child cost = parent cost + edge
cost of the re-rolled segment; every tree edge is valid; each visited region
holds exactly one node's key; keys only decrease per region; V_T is never
left; every V_A node is its region's best; parents precede children.
"""
import math

import numpy as np
import pytest

from paper_2602_02846_gb300 import scenes

A, I, T = 1, 2, 3
INF = 0xFFFFFFFFFFFFFFFF


def check_invariants(o, prob, st, prev=None):
    n = st["n_nodes"]
    assert st["parent"][0] == -1
    if n > 1:
        assert np.all(st["parent"][1:] < np.arange(1, n))
        assert np.all(st["parent"][1:] >= 0)
    for i in range(n):
        assert st["key"][i] == o.pack_key(st["cost"][i], i)
        r, _ = o.region(prob, st["x"][i])
        assert r == st["region"][i]
        assert st["key"][i] >= st["region_key"][st["region"][i]]
        if i == 0:
            continue
        p = st["parent"][i]
        ro = o.rollout(prob, st["x"][p], st["u"][i], int(st["K"][i]))
        assert ro["valid"]
        assert np.array_equal(ro["x_end"], st["x"][i])
        assert st["cost"][i] == st["cost"][p] + ro["edge_cost"]
    rk = st["region_key"]
    visited = np.nonzero(rk != np.uint64(INF))[0]
    best = {}
    for i in range(n):
        if st["key"][i] == rk[st["region"][i]]:
            assert st["region"][i] not in best
            best[st["region"][i]] = i
    assert set(best) == set(int(r) for r in visited)
    # V_A = region-best nodes only, listed in ascending id
    act = np.nonzero(st["set"] == A)[0]
    assert np.array_equal(st["VA"], act)
    for i in act:
        assert st["key"][i] == rk[st["region"][i]]
    # the solution is the least key among nodes in the goal
    gk = INF
    for i in range(n):
        if o.in_goal(prob, st["x"][i])[0]:
            gk = min(gk, int(st["key"][i]))
    assert st["goal_key"] == gk
    if prev is not None:
        assert np.all(rk <= prev["region_key"])
        pn = prev["n_nodes"]
        assert np.all(st["set"][:pn][prev["set"] == T] == T)
        assert np.array_equal(st["x"][:pn], prev["x"])


def run_checked(o, prob, iters):
    pl = o.Planner(prob)
    prev = pl.state()
    check_invariants(o, prob, prev)
    hist = [prev]
    for _ in range(iters):
        pl.iterate(1)
        st = pl.state()
        check_invariants(o, prob, st, prev)
        prev = st
        hist.append(st)
    return pl, hist


def test_di_invariants_and_solution(oracle_mod):
    o = oracle_mod
    prob = scenes.di_scene(0, grid_pos=16, tree_cap=32768)
    pl, hist = run_checked(o, prob, 10)
    last = hist[-1]
    assert last["first_solution_iter"] >= 0
    tr = pl.best_trajectory()
    # lower bound: straight line from start to the goal ball
    lb = math.dist(prob.start[:3], prob.goal_c) - prob.goal_r
    assert tr["cost"] >= lb - 1e-9
    # the returned path re-validates exactly in FP64 (its own arithmetic)
    rv = o.revalidate(prob, tr["states"], tr["controls"], tr["steps"])
    assert rv["ok"] and rv["max_seg_err"] == 0.0
    assert abs(rv["cost"] - tr["cost"]) < 1e-12
    # solution cost never increases
    costs = [o.key_cost(np.array([h["goal_key"]], np.uint64))[0] for h in hist if h["goal_key"] != INF]
    assert all(b <= a for a, b in zip(costs, costs[1:]))


def test_dubins_empty_world_invariants(oracle_mod):
    o = oracle_mod
    prob = scenes.dubins_scene(0, n_obstacles=0)
    pl, hist = run_checked(o, prob, 14)
    tr = pl.best_trajectory()
    assert tr is not None
    d = math.dist(prob.start[:3], prob.goal_c) - prob.goal_r
    assert tr["cost"] >= d / 0.3 - 1e-9          # duration >= distance / v_max
    rv = o.revalidate(prob, tr["states"], tr["controls"], tr["steps"])
    assert rv["ok"]


def test_quad_invariants_few_iterations(oracle_mod):
    o = oracle_mod
    prob = scenes.quad_scene(0, clutter=60, certify=False, tree_cap=1 << 16)
    run_checked(o, prob, 3)


def test_dubins_forest_invariants(oracle_mod):
    o = oracle_mod
    prob = scenes.dubins_scene(1)
    run_checked(o, prob, 8)


def test_capacity_rule_is_sticky(oracle_mod):
    o = oracle_mod
    prob = scenes.di_scene(0, grid_pos=16, tree_cap=300)
    pl = o.Planner(prob)
    prev = pl.state()
    full_seen = False
    for _ in range(40):
        rc = pl.iterate(1)
        st = pl.state()
        check_invariants(o, prob, st, prev)
        if st["tree_full"]:
            assert rc == o.TREE_FULL
            assert st["n_nodes"] == 300
            if full_seen:
                # no-op once full: nothing changes, iteration counter included
                assert st["iter"] == prev["iter"]
                assert np.array_equal(st["region_key"], prev["region_key"])
            full_seen = True
        prev = st
    assert full_seen


def test_fixed_and_adaptive_lambda(oracle_mod):
    """lambda = floor(t_e / |V_A|) (Eq. for the branching factor) when not fixed."""
    o = oracle_mod
    prob = scenes.di_scene(0, grid_pos=16, tree_cap=4096, lam=0)
    pl = o.Planner(prob)
    for _ in range(3):
        before = pl.state()["count_A"]
        pl.iterate(1)
        st = pl.state()
        assert st["last_lambda"] == max(1, 4096 // before)
        assert st["last_candidates"] == before * st["last_lambda"] <= 4096


def test_convergence_sanity_empty_world(oracle_mod):
    """Theorem (asymptotic delta-robust near-optimality), qualitatively: in an
    empty world the best path length approaches the straight-line bound and a
    finer grid does not end worse on the median of a few seeds."""
    o = oracle_mod
    lb = math.dist([0.05] * 3, [0.95] * 3) - 0.05
    finals = {}
    for gp in (12, 20):
        vals = []
        for seed in range(3):
            prob = scenes.di_scene(seed, n_obstacles=0, grid_pos=gp, tree_cap=1 << 15, lam=0)
            pl = o.Planner(prob)
            pl.iterate(25)
            tr = pl.best_trajectory()
            vals.append(tr["cost"] if tr else math.inf)
        finals[gp] = float(np.median(vals))
    assert finals[12] < lb * 1.15
    assert finals[20] < lb * 1.15


def test_step_functions_reproduce_the_planner(oracle_mod):
    """The per-step entry points (propagate, select_winners, prune) used by
    the GPU parity tests, chained by hand, reproduce the oracle planner's own
    iterations exactly."""
    o = oracle_mod
    prob = scenes.di_scene(2, grid_pos=16, tree_cap=4096)
    pl = o.Planner(prob)
    for _ in range(4):
        st = pl.state()
        lam = prob.lam
        rec = o.propagate(prob, st["iter"], lam, st["x"], st["cost"], st["VA"], st["count_A"])
        rk, win, kept, full = o.select_winners(st["region_key"], st["region_key"], rec["valid"],
                                               rec["region"], rec["key"], st["n_nodes"], prob.tree_cap)
        s_new, ic_new = o.prune(st["key"], st["region"], st["parent"], st["set"], st["icount"], rk, prob.i_max)
        pl.iterate(1)
        nxt = pl.state()
        n0 = st["n_nodes"]
        assert nxt["n_nodes"] == n0 + kept
        assert np.array_equal(nxt["set"][:n0], s_new)
        assert np.array_equal(nxt["icount"][:n0], ic_new)
        for rank, c in enumerate(win[:kept]):
            i = n0 + rank
            assert nxt["parent"][i] == st["VA"][rec["slot"][c] // lam]
            assert np.array_equal(nxt["x"][i], rec["x_end"][c])
            assert nxt["cost"][i] == rec["cost"][c]
            assert nxt["region"][i] == rec["region"][c]
            assert nxt["K"][i] == rec["K"][c]
            assert (int(rec["key"][c]) >> 32) == (int(nxt["key"][i]) >> 32)
            assert nxt["region_key"][rec["region"][c]] == nxt["key"][i]
