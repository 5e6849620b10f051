"""Oracle pins: compaction (Alg. 5), region argmin + V_U filter (Alg. 2/4)
and PruneNodes (Alg. 3) on hand-built inputs with hand-derived outcomes.

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
