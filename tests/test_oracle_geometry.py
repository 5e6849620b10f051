"""Oracle pins: validity (X_valid), margins, region map and goal set.

Pins: closed-box and closed-bound semantics at exact boundary points,
analytically located first collisions of straight-line motion, hand-computed
margins and clearances, hand-computed region ids at cell corners/centres,
clamping, yaw wrap-around, mixed-radix order, and the goal ball.
"""
import math

import numpy as np
import pytest

from paper_2602_02846_gb300 import scenes


def box_scene(boxes, **kw):
    p = scenes.di_scene(0, n_obstacles=0, **kw)
    return p.replace(obstacles=np.asarray(boxes, np.float32).reshape(-1, 6))


def test_closed_boxes_and_bounds(oracle_mod):
    p = box_scene([[0.25, 0.25, 0.25, 0.5, 0.5, 0.5]])
    v = np.zeros(3)
    inside_face = np.concatenate([[0.25, 0.3, 0.3], v])
    assert not oracle_mod.point_valid(p, inside_face)            # on the face: closed box
    assert oracle_mod.point_valid(p, np.concatenate([[0.2499, 0.3, 0.3], v]))
    assert not oracle_mod.point_valid(p, np.concatenate([[0.5, 0.5, 0.5], v]))  # corner
    assert oracle_mod.point_valid(p, np.concatenate([[0.5, 0.5, 0.5000001], v]))
    # workspace is closed: the boundary is valid, beyond it is not
    assert oracle_mod.point_valid(p, np.array([0.0, 1.0, 0.0, 0, 0, 0]))
    assert not oracle_mod.point_valid(p, np.array([-1e-9, 0.5, 0.5, 0, 0, 0]))
    # velocity bound |v_i| <= 1 is closed
    assert oracle_mod.point_valid(p, np.array([0.1, 0.1, 0.1, 1.0, -1.0, 0.0]))
    assert not oracle_mod.point_valid(p, np.array([0.1, 0.1, 0.1, 1.0 + 1e-12, 0.0, 0.0]))
    # NaN is invalid
    assert not oracle_mod.point_valid(p, np.array([0.1, math.nan, 0.1, 0, 0, 0]))


def test_first_collision_of_straight_line(oracle_mod):
    """Constant velocity along +x (a = 0) from x0 hits a box face at x = b:
    the first invalid step is ceil((b - x0) / (h v))."""
    h = float(np.float32(0.01))
    p = box_scene([[0.5, 0.0, 0.0, 0.6, 1.0, 1.0]])
    for x0, v in [(0.4, 0.5), (0.3, 0.9), (0.455, 0.3)]:
        r = oracle_mod.rollout(p, np.array([x0, 0.5, 0.5, v, 0, 0]), np.zeros(3, np.float32), 30)
        k_hit = math.ceil((0.5 - x0) / (h * v) - 1e-9)
        if k_hit <= 30:
            assert not r["valid"] and r["first_bad"] == k_hit
        else:
            assert r["valid"] and r["first_bad"] == -1
    # moving away never collides
    r = oracle_mod.rollout(p, np.array([0.45, 0.5, 0.5, -0.5, 0, 0]), np.zeros(3, np.float32), 30)
    assert r["valid"]


def test_margin_and_clearance_hand_values(oracle_mod):
    # box corners are FP32 inputs (0.4 -> 0.40000000596...), hence 1e-7 below
    p = box_scene([[0.4, 0.4, 0.4, 0.6, 0.6, 0.6]])
    # outside along x by 0.05, centred in y/z: Chebyshev distance 0.05; the
    # nearest other boundary is the velocity bound (|v| = 0 -> 1) and the walls
    x = np.array([0.35, 0.5, 0.5, 0.0, 0.0, 0.0])
    assert abs(oracle_mod.point_clearance(p, x) - 0.05) < 1e-7
    assert abs(oracle_mod.point_margin(p, x) - 0.05) < 1e-7
    # inside: 0.02 from the nearest face -> clearance -0.02, margin 0.02
    x = np.array([0.42, 0.5, 0.5, 0.0, 0.0, 0.0])
    assert abs(oracle_mod.point_clearance(p, x) + 0.02) < 1e-7
    assert abs(oracle_mod.point_margin(p, x) - 0.02) < 1e-7
    # near the wall and a velocity bound
    x = np.array([0.01, 0.5, 0.5, 0.995, 0.0, 0.0])
    assert abs(oracle_mod.point_clearance(p, x) - 0.005) < 1e-7
    # diagonal outside: Chebyshev = the larger gap (x: 0.1, y: 0.05)
    x = np.array([0.3, 0.35, 0.5, 0.0, 0.0, 0.0])
    assert abs(oracle_mod.point_margin(p, x) - 0.1) < 1e-7


def test_region_map_hand_values(oracle_mod):
    p = scenes.di_scene(0, n_obstacles=0)  # 8^3 x 2^3, axes p0 p1 p2 v0 v1 v2
    # origin at rest: position cells 0, velocity cells 1 ((0 - -1) * 1 = 1.0)
    r, _ = oracle_mod.region(p, np.array([0, 0, 0, 0, 0, 0]))
    assert r == ((((0 * 8 + 0) * 8 + 0) * 2 + 1) * 2 + 1) * 2 + 1
    # cell centre (0.5625 -> cell 4), corners, clamping
    r, m = oracle_mod.region(p, np.array([0.5625, 0.1875, 0.9375, -0.5, 0.5, -0.5]))
    assert r == ((((4 * 8 + 1) * 8 + 7) * 2 + 0) * 2 + 1) * 2 + 0
    assert abs(m - 0.0625) < 1e-7  # centre of a 0.125 cell (the v axes are 0.5 from 0)
    r, _ = oracle_mod.region(p, np.array([1.0, 0.125, 0.0, 1.0, -1.0, 0.999]))
    assert r == ((((7 * 8 + 1) * 8 + 0) * 2 + 1) * 2 + 0) * 2 + 1
    r, _ = oracle_mod.region(p, np.array([1.7, -0.3, 0.5, 3.0, -3.0, 0.0]))   # clamped
    assert r == ((((7 * 8 + 0) * 8 + 4) * 2 + 1) * 2 + 0) * 2 + 1
    # margin is the distance to the nearest id-changing boundary
    _, m = oracle_mod.region(p, np.array([0.126, 0.3, 0.3, 0.5, 0.5, 0.5]))
    assert abs(m - 0.001) < 1e-6


def test_region_yaw_wrap(oracle_mod):
    p = scenes.dubins_scene(0, n_obstacles=0)  # 16^3 x 4 yaw bins on [-pi, pi)
    base = np.array([0.03, 0.03, 0.03, 0.0, 0.0, 0.2])

    def yaw_cell(psi):
        x = base.copy()
        x[3] = psi
        r, m = oracle_mod.region(p, x)
        return r % 4, m
    assert yaw_cell(0.1)[0] == 2
    assert yaw_cell(-0.1)[0] == 1
    assert yaw_cell(3.0)[0] == 3
    assert yaw_cell(-3.0)[0] == 0
    # wrap: psi and psi + 2 pi k land in the same cell
    for psi in (0.3, 1.9, -2.5):
        assert yaw_cell(psi)[0] == yaw_cell(psi + 2 * math.pi)[0] == yaw_cell(psi - 4 * math.pi)[0]
    # psi = pi wraps to -pi (cell 0); margin there is ~0 (the wrap seam is a boundary)
    c, m = yaw_cell(math.pi - 1e-3)
    assert c == 3 and m < 1.1e-3
    assert yaw_cell(math.pi + 1e-3)[0] == 0
    # mixed radix: position first
    x = base.copy()
    x[:3] = [0.5, 0.25, 0.75]
    x[3] = 0.1
    r, _ = oracle_mod.region(p, x)
    assert r == ((8 * 16 + 4) * 16 + 12) * 4 + 2


def test_goal_ball(oracle_mod):
    p = scenes.di_scene(0, n_obstacles=0)
    c = np.array(p.goal_c, dtype=np.float64)
    r = float(p.goal_r)
    inside, m = oracle_mod.in_goal(p, np.concatenate([c + [r * 0.999, 0, 0], np.zeros(3)]))
    assert inside and abs(m - 0.001 * r) < 1e-9
    outside, _ = oracle_mod.in_goal(p, np.concatenate([c + [0, r * 1.001, 0], np.zeros(3)]))
    assert not outside
    on, _ = oracle_mod.in_goal(p, np.concatenate([c + [0, 0, r], np.zeros(3)]))
    assert on  # closed ball


def test_key_order(oracle_mod):
    """(cost, id) packing orders by cost, then id; tree ids < candidate ids."""
    k = [oracle_mod.pack_key(c, i) for c, i in [(0.0, 0), (0.0, 5), (0.5, 1), (0.5, 2), (1.25, 0)]]
    assert k == sorted(k)
    assert oracle_mod.pack_key(0.5, 10) < oracle_mod.pack_key(0.5, 32768 + 3)
    assert oracle_mod.key_cost(np.array([k[2]], np.uint64))[0] == np.float32(0.5)
