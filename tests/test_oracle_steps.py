"""Oracle pins: compaction (Alg. 5), region argmin + V_U filter (Alg. 2/4),
PruneNodes (Alg. 3) and UpdateTree's append (Alg. 4) on hand-built inputs
with hand-derived outcomes.

Pins: the paper's own compaction example (tests/golden), and small trees
whose expected node sets follow from reading Alg. 3 rule by rule.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A, I, T = 1, 2, 3
INF = 0xFFFFFFFFFFFFFFFF


def key(o, c, i):
    return o.pack_key(c, i)


def test_compaction_paper_example(oracle_mod):
    rows = {}
    with open(os.path.join(GOLDEN, "compaction_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows[name] = [int(v) for v in vals]
    S, Iv, cnt = oracle_mod.compact(rows["mask"])
    assert list(S) == rows["S"]
    assert list(Iv) == rows["I"]
    assert cnt == rows["count"][0]
    # the count is S[n-1] + mask[n-1]: a mask ending in 1 exposes the difference
    S, Iv, cnt = oracle_mod.compact([0, 1, 1])
    assert list(S) == [0, 0, 1] and list(Iv) == [1, 2] and cnt == 2
    S, Iv, cnt = oracle_mod.compact([])
    assert cnt == 0


def test_select_winners_min_ties_and_filter(oracle_mod):
    o = oracle_mod
    N = 100
    R = 4
    rk0 = np.array([key(o, 0.0, 0), key(o, 1.0, 1), INF, INF], np.uint64)
    # candidates in slot order: (valid, region, cost, slot)
    cands = [
        (1, 1, 1.0, 0),   # ties with tree node 1 (cost 1.0): tree id 1 < N+0 wins
        (1, 2, 0.7, 1),   # provisional best of region 2 ...
        (1, 2, 0.5, 2),   # ... beaten later: only slot 2 survives the filter
        (0, 3, 0.1, 3),   # invalid: ignored
        (1, 3, 0.9, 4),   # region 3 winner
        (1, 3, 0.9, 5),   # same cost, higher slot: loses the tie
        (1, 0, 0.2, 6),   # cannot beat the root (cost 0)
        (1, 1, 0.8, 7),   # beats tree node 1
    ]
    valid = np.array([c[0] for c in cands], np.uint8)
    reg = np.array([c[1] for c in cands], np.int32)
    keys = np.array([key(o, c[2], N + c[3]) for c in cands], np.uint64)
    rk, win, kept, full = o.select_winners(rk0, rk0, valid, reg, keys, n_nodes=2, tree_cap=N)
    assert list(win) == [2, 4, 7]
    assert kept == 3 and not full
    assert rk[0] == rk0[0]
    assert rk[1] == keys[7] and rk[2] == keys[2] and rk[3] == keys[4]


def test_select_winners_capacity(oracle_mod):
    """Room for one more node: the first winner in slot order is kept, the
    second is dropped and its region restored to the pre-iteration key."""
    o = oracle_mod
    N = 3
    rk0 = np.array([key(o, 0.0, 0), key(o, 2.0, 1), INF], np.uint64)
    valid = np.ones(2, np.uint8)
    reg = np.array([2, 1], np.int32)
    keys = np.array([key(o, 0.4, N + 0), key(o, 0.3, N + 1)], np.uint64)
    rk, win, kept, full = o.select_winners(rk0, rk0.copy(), valid, reg, keys, n_nodes=2, tree_cap=N)
    assert list(win) == [0, 1] and kept == 1 and full
    assert rk[2] == keys[0]
    assert rk[1] == rk0[1]


def _tree():
    """root 0 (region 0) -> 1 (region 1) -> 2 (region 2) -> 3 (region 3);
    root -> 4 (region 4)."""
    parent = np.array([-1, 0, 1, 2, 0], np.int32)
    region = np.array([0, 1, 2, 3, 4], np.int32)
    return parent, region


def test_prune_terminal_and_inactive(oracle_mod):
    o = oracle_mod
    parent, region = _tree()
    costs = [0.0, 0.3, 0.6, 0.9, 0.2]
    keys = np.array([key(o, c, i) for i, c in enumerate(costs)], np.uint64)
    rk = keys.copy()  # every node best in its region
    rk[1] = key(o, 0.25, 50)  # node 1's region improved by someone else
    sets = np.full(5, A, np.uint8)
    ic = np.zeros(5, np.uint8)
    s, c = o.prune(keys, region, parent, sets, ic, rk, i_max=3)
    # 1: dominated -> V_T; 2, 3: best but an ancestor is dominated -> V_I;
    # 0 and 4: best with clean ancestry -> stay in V_A (no rule applies)
    assert list(s) == [A, T, I, I, A]
    assert list(c) == [0, 0, 0, 0, 0]


def test_prune_reactivation_after_imax(oracle_mod):
    o = oracle_mod
    parent, region = _tree()
    costs = [0.0, 0.3, 0.6, 0.9, 0.2]
    keys = np.array([key(o, c, i) for i, c in enumerate(costs)], np.uint64)
    rk = keys.copy()
    rk[1] = key(o, 0.25, 50)
    sets = np.array([A, T, I, I, A], np.uint8)
    ic = np.zeros(5, np.uint8)
    i_max = 2
    history = []
    for _ in range(4):
        sets, ic = o.prune(keys, region, parent, sets, ic, rk, i_max=i_max)
        history.append((list(sets), list(ic)))
    # each pass increments I_count of best V_I nodes; on the pass where it
    # exceeds I_max (third) they return to V_A and then stay (rule 2)
    assert history[0] == ([A, T, I, I, A], [0, 0, 1, 1, 0])
    assert history[1] == ([A, T, I, I, A], [0, 0, 2, 2, 0])
    assert history[2] == ([A, T, A, A, A], [0, 0, 3, 3, 0])
    assert history[3] == ([A, T, A, A, A], [0, 0, 3, 3, 0])
    # a reactivated node that later loses its region goes to V_T (rule 3)
    rk[3] = key(o, 0.8, 60)
    sets, ic = o.prune(keys, region, parent, sets, ic, rk, i_max=i_max)
    assert list(sets) == [A, T, A, T, A]


def test_prune_inactive_not_best_goes_terminal_and_t_is_permanent(oracle_mod):
    o = oracle_mod
    parent, region = _tree()
    parent[4] = 2  # node 4 hangs below node 2
    costs = [0.0, 0.3, 0.6, 0.9, 0.2]
    keys = np.array([key(o, c, i) for i, c in enumerate(costs)], np.uint64)
    rk = keys.copy()
    rk[2] = key(o, 0.5, 70)  # node 2 (in V_I) no longer best
    rk[4] = key(o, 0.1, 71)  # node 4 was terminal already; its region keeps improving
    sets = np.array([A, A, I, A, T], np.uint8)
    ic = np.array([0, 0, 1, 0, 0], np.uint8)
    s, c = o.prune(keys, region, parent, sets, ic, rk, i_max=5)
    assert list(s) == [A, A, T, I, T]
    assert list(c) == [0, 0, 1, 0, 0]
    # even if the region's best were restored (node 4 best again, below the
    # dominated node 2), V_T is never left
    rk[4] = keys[4]
    s, c = o.prune(keys, region, parent, s, c, rk, i_max=5)
    assert s[4] == T


def test_prune_ancestor_chain_is_strict_and_reaches_root(oracle_mod):
    """Only strict ancestors count; a dominated great-grandparent suffices."""
    o = oracle_mod
    parent, region = _tree()
    keys = np.array([key(o, c, i) for i, c in enumerate([0.0, 0.3, 0.6, 0.9, 0.2])], np.uint64)
    rk = keys.copy()
    sets = np.full(5, A, np.uint8)
    ic = np.zeros(5, np.uint8)
    # node 3 itself best and clean ancestry: unchanged
    s, _ = o.prune(keys, region, parent, sets, ic, rk, i_max=3)
    assert list(s) == [A, A, A, A, A]
    # dominate node 1: the grandchild 3 becomes inactive through 2
    rk[1] = key(o, 0.1, 99)
    s, _ = o.prune(keys, region, parent, sets, ic, rk, i_max=3)
    assert list(s) == [A, T, I, I, A]


def _append_case(o):
    """A 2-node tree (DI dimensions) and two kept winners: slot order gives
    node ids 2 and 3; only the second, the dearer one, ends in the goal set."""
    from paper_2602_02846_gb300 import scenes
    prob = scenes.di_scene(0)
    n, m, N, R = prob.n, prob.m, 8, 16
    tree = dict(x=np.zeros((N, n)), u=np.zeros((N, m), np.float32), K=np.zeros(N, np.int32),
                parent=np.full(N, -1, np.int32), cost=np.zeros(N), key=np.full(N, INF, np.uint64),
                region=np.zeros(N, np.int32), set=np.zeros(N, np.uint8), icount=np.zeros(N, np.uint8))
    tree["key"][0] = key(o, 0.0, 0)
    tree["key"][1] = key(o, 0.75, 1)
    tree["region"][:2] = [3, 5]
    tree["set"][:2] = [A, I]
    tree["icount"][1] = 4
    rk = np.full(R, INF, np.uint64)
    rk[3], rk[5] = tree["key"][0], tree["key"][1]
    cand = dict(x=np.arange(2 * n, dtype=np.float64).reshape(2, n), u=np.array([[1, 2, 3], [4, 5, 6]], np.float32),
                K=np.array([7, 9], np.int32), parent=np.array([0, 1], np.int32), cost=np.array([0.25, 0.5]),
                region=np.array([5, 7], np.int32), goal=np.array([0, 1], np.uint8))
    return prob, tree, rk, cand


def test_append_rows_keys_and_solution(oracle_mod):
    o = oracle_mod
    prob, tree, rk, cand = _append_case(o)
    t, rk2, gk, first = o.append(prob, 2, cand, tree, rk, INF)
    for k, i in enumerate((2, 3)):
        assert np.array_equal(t["x"][i], cand["x"][k]) and np.array_equal(t["u"][i], cand["u"][k])
        assert t["K"][i] == cand["K"][k] and t["parent"][i] == cand["parent"][k]
        assert t["cost"][i] == cand["cost"][k] and t["region"][i] == cand["region"][k]
        assert t["key"][i] == key(o, float(cand["cost"][k]), i)  # (cost, id): the node's own id
        assert t["set"][i] == A and t["icount"][i] == 0
    # each winner's key becomes its region's key (region 5 changes hands)
    assert rk2[5] == key(o, 0.25, 2) and rk2[7] == key(o, 0.5, 3)
    assert rk2[3] == rk[3] and np.all(np.delete(rk2, [5, 7]) == np.delete(rk, [5, 7]))
    # the untouched nodes keep their rows
    assert t["key"][1] == tree["key"][1] and t["set"][1] == I and t["icount"][1] == 4
    # the appended goal node is the solution (not the cheaper non-goal one), the first one
    assert gk == key(o, 0.5, 3) and first
    # a better solution already held is kept and is not a first
    best = key(o, 0.1, 1)
    _, _, gk, first = o.append(prob, 2, cand, tree, rk, best)
    assert gk == best and not first


def test_append_then_planner_iteration_agree(oracle_mod):
    """One planner iteration equals its steps composed by hand: propagate,
    select winners, prune, append."""
    from paper_2602_02846_gb300 import scenes
    o = oracle_mod
    prob = scenes.di_scene(1, grid_pos=16, tree_cap=4096)
    pl = o.Planner(prob)
    pl.iterate(3)
    s0 = pl.state()
    n0 = s0["n_nodes"]
    it, lam = s0["iter"], int(prob.lam)
    pr = o.propagate(prob, it, lam, s0["x"][:n0], s0["cost"][:n0], s0["VA"], s0["count_A"])
    rk, win, kept, full = o.select_winners(s0["region_key"], s0["region_key"], pr["valid"],
                                           np.where(pr["valid"] == 1, pr["region"], 0), pr["key"], n0,
                                           int(prob.tree_cap))
    st, ic = o.prune(s0["key"][:n0], s0["region"][:n0], s0["parent"][:n0], s0["set"][:n0], s0["icount"][:n0], rk,
                     prob.i_max)
    ws = win[:kept]
    cand = dict(x=pr["x_end"][ws], u=pr["u"][ws], K=pr["K"][ws], parent=np.asarray(s0["VA"])[ws // lam],
                cost=pr["cost"][ws], region=pr["region"][ws], goal=pr["in_goal"][ws])
    n1 = n0 + kept

    def rows(a):  # the first n0 rows, room for the appended ones after them
        a = np.asarray(a)
        return np.concatenate([a, np.zeros((kept,) + a.shape[1:], a.dtype)])
    tree = {name: rows(s0[name]) for name in ("x", "u", "K", "parent", "cost", "key", "region")}
    tree["set"], tree["icount"] = rows(st), rows(ic)
    t, rk2, gk, _ = o.append(prob, n0, cand, tree, rk, s0["goal_key"])
    pl.iterate(1)
    s1 = pl.state()
    assert s1["n_nodes"] == n1 and not full and kept > 0
    for name in ("x", "u", "K", "parent", "key", "region", "set", "icount"):
        assert np.array_equal(np.asarray(s1[name])[:n1], t[name][:n1]), name
    assert np.array_equal(s1["region_key"], rk2) and s1["goal_key"] == gk

