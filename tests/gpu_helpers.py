"""Helpers for the GPU parity tests: run one iteration of the CUDA planner
phase by phase and compare each phase with the FP64 oracle on the same
inputs.

Tolerances (stated once, used everywhere):
  * decisions (regions, winners, node sets, ids, counts) are compared
    bit-exactly when both sides see identical inputs; the oracle's winner
    selection, append and prune are fed the GPU's candidate keys;
  * propagated end states: |gpu - oracle| / max(1, |oracle|) <= 1e-4 per
    component (FP32 integration against FP64, one segment);
  * validity verdicts, region ids and goal tests must agree except where the
    oracle finds a checked point within 1e-4 of a face, a bound or a cell
    boundary; such slots are counted and reported.
"""
import numpy as np

import oracle

REL_TOL = 1e-4
NEAR = 1e-4
A, I, T = 1, 2, 3


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def oracle_inputs(arr):
    return arr["x"].astype(np.float64), oracle.key_cost(arr["key"]).astype(np.float64)


def records_host(rec, n, m, ns):
    return dict(
        valid=rec["valid"][:ns].cpu().numpy(),
        region=rec["region"][:ns].cpu().numpy(),
        key=rec["key"][:ns].cpu().numpy().view(np.uint64),
        K=rec["K"][:ns].cpu().numpy(),
        x=rec["x"].view(n, -1)[:, :ns].T.cpu().numpy(),
        u=rec["u"].view(m, -1)[:, :ns].T.cpu().numpy(),
    )


def compare_propagate(prob, g, o, slots=None):
    """GPU records g vs oracle propagate o (same slots).  Returns a report."""
    if slots is not None:
        g = {k: v[slots] for k, v in g.items()}
    assert np.array_equal(g["K"], o["K"]), "K differs"
    assert np.array_equal(g["u"].view(np.uint32), o["u"].view(np.uint32)), "controls differ"
    near_v = o["vmargin"] < NEAR
    vmis = (g["valid"] != o["valid"])
    assert np.all(~vmis | near_v), "validity differs away from any boundary: %s" % np.nonzero(vmis & ~near_v)[0][:10]
    both = (g["valid"] == 1) & (o["valid"] == 1)
    err = rel_err(g["x"][both], o["x_end"][both])
    max_err = float(err.max()) if err.size else 0.0
    assert max_err <= REL_TOL, "end state error %.3g" % max_err
    near_r = o["rmargin"][both] < NEAR
    rmis = g["region"][both] != o["region"][both]
    assert np.all(~rmis | near_r), "region differs away from a cell boundary"
    gcost = oracle.key_cost(g["key"][both]).astype(np.float64)
    cerr = rel_err(gcost, o["cost"][both])
    assert cerr.size == 0 or cerr.max() <= REL_TOL, "cost error %.3g" % cerr.max()
    gid = (g["key"][both] & np.uint64(0xFFFFFFFF))
    oid = (o["key"][both] & np.uint64(0xFFFFFFFF))
    assert np.array_equal(gid, oid), "candidate ids differ"
    return dict(slots=int(len(g["K"])), valid=int(g["valid"].sum()), both_valid=int(both.sum()),
                validity_exempt=int((vmis & near_v).sum()), region_exempt=int((rmis & near_r).sum()),
                max_state_err=max_err, max_cost_err=float(cerr.max()) if cerr.size else 0.0)


def step_phases(pl, prob, check_append=True, sample_slots=None, seed=0):
    """Runs one iteration phase by phase on the GPU and checks every phase
    against the oracle.  With ``sample_slots`` the oracle re-rolls that many
    sampled slots (plus the first and last) instead of every slot; every other
    phase is still checked in full.  Returns the report dict."""
    import torch
    n, m = prob.n, prob.m
    before = pl.arrays()
    rec = pl.make_records()
    pl.debug_step("begin")
    pl.debug_step("propagate", rec)
    h = pl.header()
    ns, lam, it = int(h.n_slots), int(h.lam), int(h.iter)
    N = pl.layout().N
    g = records_host(rec, n, m, ns)
    tx, tc = oracle_inputs(before)
    if sample_slots is not None and sample_slots < ns:
        rng = np.random.default_rng(seed)
        sl = np.unique(np.concatenate([rng.integers(0, ns, size=sample_slots), [0, ns - 1]]))
        o = oracle.propagate(prob, it, lam, tx, tc, before["VA"], h.count_A, slots=sl)
        rep = compare_propagate(prob, g, o, slots=sl)
    else:
        o = oracle.propagate(prob, it, lam, tx, tc, before["VA"], h.count_A)
        rep = compare_propagate(prob, g, o)
    # region argmin: the GPU's region keys after propagate equal the min over
    # its own candidate keys (atomicMin) -- bit-exact
    mid = pl.arrays()
    rk_ref, win, kept, full = oracle.select_winners(before["region_key"], before["region_key"], g["valid"],
                                                    np.where(g["valid"] == 1, g["region"], 0), g["key"],
                                                    before["n_nodes"], N)
    # before the capacity restore, the oracle's region keys equal the GPU's
    rk_pre, _, _, _ = oracle.select_winners(before["region_key"], before["region_key"], g["valid"],
                                            np.where(g["valid"] == 1, g["region"], 0), g["key"], 0, 2 ** 31 - 1)
    assert np.array_equal(mid["region_key"], rk_pre), "region argmin differs"
    pl.debug_step("mark")
    pl.debug_step("scan")
    h = pl.header()
    W = int(h.n_win)
    gw = pl.win_slots(W)
    assert W == len(win), "winner count differs: gpu %d oracle %d" % (W, len(win))
    assert np.array_equal(gw, win.astype(np.int32)), "winner slots differ"
    pl.debug_step("append")
    after = pl.arrays(n_nodes=before["n_nodes"] + kept)
    h = pl.header()
    assert int(h.n_kept) == kept
    assert (int(h.status) == 4) == full, "capacity rule differs"
    assert np.array_equal(after["region_key"], rk_ref_with_ids(rk_ref, g, win, kept, before["n_nodes"], N))
    if check_append and kept:
        n0 = before["n_nodes"]
        ids = np.arange(n0, n0 + kept)
        ws = win[:kept]
        # UpdateTree (Alg. 4) by the oracle on the GPU's winning candidates:
        # rows, keys, region keys and the solution key
        goal, amb = np.zeros(kept, np.uint8), 0
        for k, w in enumerate(ws):
            inside, margin = oracle.in_goal(prob, g["x"][w].astype(np.float64))
            goal[k] = 1 if inside else 0
            amb += 1 if margin < NEAR else 0
        cand = dict(x=g["x"][ws].astype(np.float64), u=g["u"][ws], K=g["K"][ws], parent=before["VA"][ws // lam],
                    cost=oracle.key_cost(g["key"][ws]).astype(np.float64), region=g["region"][ws], goal=goal)

        def rows(a):
            a = np.asarray(a)[:n0]
            return np.concatenate([a, np.zeros((kept,) + a.shape[1:], a.dtype)])
        tree = {name: rows(before[name]) for name in ("x", "u", "K", "parent", "key", "region", "set", "icount")}
        tree["cost"] = rows(oracle.key_cost(before["key"]).astype(np.float64))
        t, rk_o, gk_o, _ = oracle.append(prob, n0, cand, tree, rk_ref, before["goal_key"])
        assert np.array_equal(after["region_key"], rk_o), "region keys after append differ from the oracle's"
        assert np.array_equal(after["parent"][ids], t["parent"][ids]), "parents differ"
        assert np.array_equal(after["K"][ids], t["K"][ids]), "K differs"
        assert np.array_equal(after["u"][ids].view(np.uint32), t["u"][ids].view(np.uint32)), "controls differ"
        # re-materialised winners are bit-identical to the propagate records
        assert np.array_equal(after["x"][ids].view(np.uint32), g["x"][ws].view(np.uint32)), "re-materialised state differs"
        assert np.array_equal(after["key"][ids], t["key"][ids]), "keys differ"
        assert np.array_equal(after["region"][ids], t["region"][ids])
        assert np.array_equal(after["set"][ids], t["set"][ids]) and np.array_equal(after["icount"][ids],
                                                                                   t["icount"][ids])
        # solution: least key among appended goal nodes (oracle goal test in FP64)
        if amb == 0:
            assert int(pl.header().goal_key) == gk_o, "solution key differs"
        rep["goal_exempt"] = amb
    # prune: oracle Alg. 3 on the same (pre-append) nodes and region keys
    s_ref, ic_ref = oracle.prune(before["key"], before["region"], before["parent"], before["set"],
                                 before["icount"], after["region_key"], prob.i_max)
    pl.debug_step("prune")
    pr = pl.arrays(n_nodes=before["n_nodes"] + kept)
    n0 = before["n_nodes"]
    assert np.array_equal(pr["set"][:n0], s_ref), "node sets differ after prune"
    assert np.array_equal(pr["icount"][:n0], ic_ref), "inactivity counters differ after prune"
    pl.debug_step("end")
    fin = pl.arrays()
    expect_va = np.nonzero(fin["set"] == A)[0].astype(np.int32)
    # the memoised "dominated" bit equals key(i) != key(region(i)) on every node
    dom_bit = (fin["set_raw"] & 8) != 0
    dom_key = fin["key"] != fin["region_key"][fin["region"]]
    assert np.array_equal(dom_bit, dom_key), "dominated bit out of step with the region keys"
    assert fin["n_nodes"] == n0 + kept
    assert np.array_equal(fin["VA"], expect_va), "next V_A differs from the ascending active ids"
    assert fin["iter"] == it + 1
    rep.update(winners=W, kept=kept, full=full, n_nodes=int(fin["n_nodes"]), count_A=int(fin["count_A"]))
    return rep


def rk_ref_with_ids(rk_ref, g, win, kept, n0, N):
    """Oracle region keys after append: kept winners carry their new ids."""
    rk = rk_ref.copy()
    for rank in range(kept):
        s = win[rank]
        r = g["region"][s]
        rk[r] = (g["key"][s] & np.uint64(0xFFFFFFFF00000000)) | np.uint64(n0 + rank)
    return rk


def check_tree_fp64(prob, a, created=None, lam_at=None, max_nodes=None):
    """Oracle-anchored invariants of a GPU tree (``a`` from Planner.arrays()).

    Every edge is re-rolled by the oracle in FP64 from the parent's stored
    state with the stored control and step count (Alg. 2): the segment is
    valid, reaches the stored state within REL_TOL, and the node's cost is
    the parent's plus the edge cost (Assumption 1).  The stored region is the
    oracle's region of the stored state (the FP32 region map of both sides,
    bit-exact), the key packs (FP32 cost, id), each visited region's key is
    held by exactly one node of that region, V_A nodes are region-best and
    V_T nodes are dominated, and the solution key is the least key among the
    goal nodes.  With ``created`` (iteration that appended each node) and
    ``lam_at`` (lambda of each iteration), every node's control and step
    count must be the Philox draw (iteration, parent, s) for some sample
    s < lambda, and each iteration's nodes must come in ascending (parent,
    s) order (Alg. 4's append order).  Segments whose oracle re-roll passes
    within NEAR of a face or bound are exempt from the validity check and
    counted.  Returns a report."""
    n = int(a["n_nodes"])
    m = max_nodes if max_nodes is not None else n
    ids = np.arange(n, dtype=np.int64)
    par = a["parent"][:n].astype(np.int64)
    assert par[0] == -1
    assert np.all(par[1:] >= 0) and np.all(par[1:] < ids[1:]), "parents must precede children"
    key = a["key"][:n]
    assert np.array_equal(key & np.uint64(0xFFFFFFFF), ids.astype(np.uint64)), "key ids"
    cost = oracle.key_cost(key).astype(np.float64)
    x = a["x"][:n].astype(np.float64)
    r0, _ = oracle.region(prob, x[0])
    assert r0 == a["region"][0]
    worst, exempt, draws_checked = 0.0, 0, 0
    last_order, draws = {}, {}
    for i in range(1, min(n, m)):
        p = int(par[i])
        ro = oracle.rollout(prob, x[p], a["u"][i], int(a["K"][i]))
        if not ro["valid"]:
            assert ro["margin"] < NEAR, "edge %d invalid away from any boundary" % i
            exempt += 1
        worst = max(worst, float(rel_err(a["x"][i], ro["x_end"]).max()))
        assert abs(cost[i] - (cost[p] + ro["edge_cost"])) <= REL_TOL * max(1.0, cost[i]), "cost of node %d" % i
        reg, _ = oracle.region(prob, x[i])
        assert reg == a["region"][i], "region of node %d" % i
        if created is not None:
            t = int(created[i])
            if (t, p) not in draws:
                # every sample of parent p at iteration t (the oracle's Alg. 2 with V_A = [p])
                o = oracle.propagate(prob, t, int(lam_at[t]), x, cost, np.array([p], np.int32), 1)
                draws[(t, p)] = (o["u"].view(np.uint32), o["K"])
            du, dk = draws[(t, p)]
            hits = np.nonzero((dk == int(a["K"][i])) &
                              np.all(du == np.asarray(a["u"][i], np.float32).view(np.uint32), axis=1))[0]
            assert hits.size, "node %d: (u, K) is no Philox draw of its parent at iteration %d" % (i, t)
            prev = last_order.get(t, (-1, -1))
            later = hits[[(p, int(h)) > prev for h in hits]]
            assert later.size, "iteration %d appends out of slot order at node %d" % (t, i)
            last_order[t] = (p, int(later[0]))
            draws_checked += 1
    assert worst <= REL_TOL, "end state error %.3g" % worst
    rk = a["region_key"]
    reg = a["region"][:n].astype(np.int64)
    assert np.all(key >= rk[reg]), "a node's key below its region's key"
    visited = np.nonzero(rk != np.uint64(oracle.KEY_INF))[0]
    owner = (rk[visited] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.all(owner < n) and np.array_equal(reg[owner], visited), "region key owners"
    assert np.array_equal(key[owner], rk[visited])
    setb = a["set"][:n]
    assert np.all(key[setb == A] == rk[reg[setb == A]]), "V_A node not its region's best"
    assert np.all(key[setb == T] > rk[reg[setb == T]]), "V_T node holds its region"
    goal_key = int(a["goal_key"])
    goal_exempt = 0
    if goal_key != oracle.KEY_INF:
        gid = goal_key & 0xFFFFFFFF
        inside, margin = oracle.in_goal(prob, x[gid])
        assert inside or margin < NEAR, "solution node outside the goal ball"
        assert int(key[gid]) == goal_key
    for i in range(min(n, m)):
        inside, margin = oracle.in_goal(prob, x[i])
        if margin < NEAR:
            goal_exempt += 1
        elif inside:
            assert goal_key != oracle.KEY_INF and int(key[i]) >= goal_key, "goal node %d beats the solution" % i
    return dict(nodes=n, checked=min(n, m), max_state_err=worst, validity_exempt=exempt, goal_exempt=goal_exempt,
                draws_checked=draws_checked)


def revalidate_trajectory(prob, tr):
    """The oracle's FP64 re-validation of a returned trajectory (Sec. III)."""
    rv = oracle.revalidate(prob, tr["states"].astype(np.float64), tr["controls"], tr["steps"])
    assert rv["ok"], rv
    assert abs(rv["cost"] - tr["cost"]) <= REL_TOL * max(1.0, tr["cost"]), (rv["cost"], tr["cost"])
    return rv
