"""Oracle pins: FP64 re-validation of a returned trajectory and the
trajectory the oracle's own planner returns.

A solution (Sec. III) follows the dynamics x' = f(x, u), stays in X_valid
(workspace, state bounds, outside every closed obstacle box) and ends in the
goal set.  The re-validation must therefore reject a trajectory that breaks
any one of these, and accept one that keeps all of them.

The trajectories here are double-integrator flights built by hand: straight
flights at constant velocity (a = 0) and one constant-acceleration flight,
whose checked points follow forward Euler, p_(k+1) = p_k + h v_k and
v_(k+1) = v_k + h a.  So every expected verdict, clearance, goal slack and
cost below is known without running the oracle:
- a thin box that holds exactly one checked point (clearance -1e-3);
- a box face 5e-5 inside a checked point (within the -1e-4 tolerance);
- a flight that leaves the workspace (clearance -0.05);
- a flight whose speed passes the bound |v_i| <= 1 (clearance -0.05);
- a start inside a box;
- a flight that stops 1e-3 short of the goal ball;
- a stored state moved by 1e-3 (dynamically inconsistent) and by 1e-6
  (within the 1e-4 tolerance).

The returned trajectory (Alg. 1's solution, the parent walk from the goal
node) is checked against the tree arrays walked by hand.
"""
import math

import numpy as np
import pytest

from paper_2602_02846_gb300 import scenes


def di_world(boxes=(), goal_c=(0.95, 0.95, 0.95), goal_r=0.05):
    p = scenes.di_scene(0, n_obstacles=0)
    return p.replace(obstacles=np.asarray(boxes, np.float32).reshape(-1, 6),
                     goal_c=[scenes.f32(c) for c in goal_c], goal_r=scenes.f32(goal_r))


def flight(prob, p0, v0, a=(0.0, 0.0, 0.0), segs=3, K=10):
    """Forward-Euler states of a double integrator under a constant control."""
    h = prob.h
    x = np.array(list(p0) + list(v0), np.float64)
    states = [x.copy()]
    for _ in range(segs):
        for _ in range(K):
            nx = x.copy()
            for i in range(3):
                nx[i] = x[i] + h * x[3 + i]
                nx[3 + i] = x[3 + i] + h * float(np.float32(a[i]))
            x = nx
        states.append(x.copy())
    controls = np.tile(np.asarray(a, np.float32), (segs, 1))
    steps = np.full(segs, K, np.int32)
    return np.asarray(states), controls, steps


def point_x(prob, x0, v, k):
    """x coordinate of checked point k of a straight flight along x."""
    x = x0
    for _ in range(k):
        x = x + prob.h * v
    return x


def test_revalidate_accepts_valid_flight(oracle_mod):
    o = oracle_mod
    probe = di_world()
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.5, 0.0, 0.0))
    end = st[-1, :3]
    prob = di_world(goal_c=(end[0] + 0.03, 0.5, 0.5))
    rv = o.revalidate(prob, st, ct, sp)
    assert rv["ok"], rv
    assert rv["max_seg_err"] == 0.0 and rv["openloop_err"] == 0.0
    # nearest constraint: the workspace face x = 0, 0.1 from the start (speed and y, z leave 0.5)
    assert abs(rv["min_clearance"] - 0.1) < 1e-12
    assert abs(rv["goal_slack"] - 0.02) < 1e-6
    # path length: 30 steps of h * 0.5
    assert abs(rv["cost"] - 30 * prob.h * 0.5) < 1e-12


def test_revalidate_rejects_one_point_in_thin_box(oracle_mod):
    o = oracle_mod
    probe = di_world()
    x17 = point_x(probe, 0.1, 0.5, 17)       # segment 2, step 7
    box = [x17 - 1e-3, 0.4, 0.4, x17 + 1e-3, 0.6, 0.6]
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.5, 0.0, 0.0))
    prob = di_world(boxes=[box], goal_c=(st[-1, 0], 0.5, 0.5))
    # the neighbouring checked points lie 4e-3 outside the box: only point 17 is inside
    for k in (16, 18):
        assert abs(point_x(probe, 0.1, 0.5, k) - x17) > 3.9e-3
    rv = o.revalidate(prob, st, ct, sp)
    assert not rv["ok"], rv
    assert abs(rv["min_clearance"] + 1e-3) < 1e-6
    assert rv["max_seg_err"] == 0.0        # the stored states are the dynamics' own


def test_revalidate_tolerates_face_within_1e4(oracle_mod):
    o = oracle_mod
    probe = di_world()
    x17 = point_x(probe, 0.1, 0.5, 17)
    box = [x17 - 5e-5, 0.4, 0.4, x17 + 0.002, 0.6, 0.6]   # point 17 is 5e-5 inside the lower x face
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.5, 0.0, 0.0))
    prob = di_world(boxes=[box], goal_c=(st[-1, 0], 0.5, 0.5))
    rv = o.revalidate(prob, st, ct, sp)
    assert rv["ok"], rv
    assert -1e-4 < rv["min_clearance"] < 0.0
    assert abs(rv["min_clearance"] + 5e-5) < 1e-6


def test_revalidate_rejects_leaving_workspace(oracle_mod):
    o = oracle_mod
    probe = di_world()
    st, ct, sp = flight(probe, (0.9, 0.5, 0.5), (0.5, 0.0, 0.0))
    prob = di_world(goal_c=(st[-1, 0], 0.5, 0.5))
    assert st[-1, 0] > 1.0
    rv = o.revalidate(prob, st, ct, sp)
    assert not rv["ok"], rv
    assert abs(rv["min_clearance"] - (1.0 - st[-1, 0])) < 1e-12
    assert abs(rv["min_clearance"] + 0.05) < 1e-6


def test_revalidate_rejects_speed_bound(oracle_mod):
    o = oracle_mod
    probe = di_world()
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.95, 0.0, 0.0), a=(1.0, 0.0, 0.0), segs=1, K=10)
    prob = di_world(goal_c=(st[-1, 0], 0.5, 0.5))
    v_end = st[-1, 3]
    assert abs(v_end - 1.05) < 1e-6
    rv = o.revalidate(prob, st, ct, sp)
    assert not rv["ok"], rv
    assert abs(rv["min_clearance"] - (1.0 - v_end)) < 1e-12


def test_revalidate_rejects_start_in_box(oracle_mod):
    o = oracle_mod
    probe = di_world()
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.5, 0.0, 0.0))
    box = [0.1 - 5e-4, 0.45, 0.45, 0.1 + 5e-4, 0.55, 0.55]    # holds the start only
    prob = di_world(boxes=[box], goal_c=(st[-1, 0], 0.5, 0.5))
    assert point_x(probe, 0.1, 0.5, 1) > 0.1 + 5e-4 + 4e-3
    rv = o.revalidate(prob, st, ct, sp)
    assert not rv["ok"], rv
    assert abs(rv["min_clearance"] + 5e-4) < 1e-6


def test_revalidate_rejects_missing_the_goal(oracle_mod):
    o = oracle_mod
    probe = di_world()
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.5, 0.0, 0.0))
    end_x = st[-1, 0]
    prob = di_world(goal_c=(end_x + 0.051, 0.5, 0.5), goal_r=0.05)
    d = math.dist(st[-1, :3], prob.goal_c)
    rv = o.revalidate(prob, st, ct, sp)
    assert not rv["ok"], rv
    assert abs(rv["goal_slack"] - (prob.goal_r - d)) < 1e-12
    assert abs(rv["goal_slack"] + 1e-3) < 1e-6
    # the same flight one step further along would end inside: the verdict follows the last stored state
    prob_in = di_world(goal_c=(end_x + 0.049, 0.5, 0.5), goal_r=0.05)
    rv_in = o.revalidate(prob_in, st, ct, sp)
    assert rv_in["ok"] and abs(rv_in["goal_slack"] - 1e-3) < 1e-6


def test_revalidate_rejects_inconsistent_stored_state(oracle_mod):
    o = oracle_mod
    probe = di_world()
    st, ct, sp = flight(probe, (0.1, 0.5, 0.5), (0.5, 0.0, 0.0))
    prob = di_world(goal_c=(st[-1, 0], 0.5, 0.5))
    bad = st.copy()
    bad[2, 1] += 1e-3          # the end of segment 2 moved sideways: no control of the segment reaches it
    rv = o.revalidate(prob, bad, ct, sp)
    assert not rv["ok"], rv
    assert abs(rv["max_seg_err"] - 1e-3) < 1e-9
    assert abs(rv["openloop_err"] - 1e-3) < 1e-9
    assert rv["min_clearance"] > 0.09       # nothing else is wrong with it
    small = st.copy()
    small[2, 1] += 1e-6        # within the 1e-4 relative tolerance
    rv2 = o.revalidate(prob, small, ct, sp)
    assert rv2["ok"], rv2
    assert abs(rv2["max_seg_err"] - 1e-6) < 1e-9


def test_best_trajectory_is_the_parent_walk(oracle_mod):
    """The oracle's returned trajectory equals the parent walk from the goal
    node through the tree arrays, and re-rolls exactly in FP64."""
    o = oracle_mod
    prob = scenes.di_scene(0, grid_pos=16, tree_cap=32768)
    pl = o.Planner(prob)
    pl.iterate(10)
    st = pl.state()
    assert st["goal_key"] != o.KEY_INF
    gid = int(st["goal_key"]) & 0xFFFFFFFF
    chain = [gid]
    while st["parent"][chain[-1]] >= 0:
        chain.append(int(st["parent"][chain[-1]]))
    chain = chain[::-1]
    assert chain[0] == 0
    tr = pl.best_trajectory()
    L = len(chain) - 1
    assert len(tr["steps"]) == L and tr["states"].shape == (L + 1, prob.n)
    assert np.array_equal(tr["states"][0], np.asarray(prob.start, np.float64))
    assert np.array_equal(tr["states"], st["x"][chain])
    assert np.array_equal(tr["controls"], st["u"][chain[1:]])
    assert np.array_equal(tr["steps"], st["K"][chain[1:]])
    assert tr["cost"] == st["cost"][gid]
    rv = o.revalidate(prob, tr["states"], tr["controls"], tr["steps"])
    assert rv["ok"] and rv["max_seg_err"] == 0.0 and rv["openloop_err"] == 0.0
    assert abs(rv["cost"] - tr["cost"]) < 1e-12
