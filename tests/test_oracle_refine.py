"""Pins of the oracle's refinement objective and its reverse-mode gradient
(the reference for the adjoint kernel): box distances by hand, the effort
cost and its gradient in closed form, an exact thrust gradient at hover (RK4
integrates the quadratic climb exactly), FP64 central differences of the
objective on cluttered cases, and the open-loop re-validation."""
import math

import numpy as np

from paper_2602_02846_gb300 import scenes

_Q = scenes.quad_scene(0, clutter=-1)
MASS, G, TAU_MAX = float(_Q.param[0]), float(_Q.param[1]), float(_Q.param[5])  # FP32-rounded, as the oracle sees them
MG = MASS * G


def _spec(**kw):
    s = dict(w_obs=1.0, beta=200.0, margin=0.01, w_goal=10.0, goal=[0.95, 0.5, 0.5], w_effort=1.0)
    s.update(kw)
    return s


def test_box_distance_hand_values(oracle_mod):
    box = [0.0, 0.0, 0.0, 1.0, 1.0, 1.0]
    cases = [([2.0, 0.5, 0.5], 1.0, [1, 0, 0]), ([-0.5, 0.5, 0.5], 0.5, [-1, 0, 0]),
             ([2.0, 2.0, 0.5], math.sqrt(2.0), [1 / math.sqrt(2), 1 / math.sqrt(2), 0]),
             ([2.0, 3.0, -2.0], math.sqrt(1 + 4 + 4), [1 / 3, 2 / 3, -2 / 3]),
             ([0.5, 0.5, 0.1], -0.1, [0, 0, -1]), ([0.5, 0.95, 0.5], -0.05, [0, 1, 0]),
             ([0.5, 0.5, 1.0], 0.0, None)]
    for p, d, g in cases:
        dd, gg = oracle_mod.box_distance(box, p)
        assert abs(dd - d) < 1e-12, (p, dd, d)
        if g is not None:
            assert np.allclose(gg, g, atol=1e-12), (p, gg, g)


def _hover_case(K, T, tau=(0.0, 0.0, 0.0)):
    prob = scenes.quad_scene(0, clutter=-1)
    x0 = np.array(prob.start, dtype=np.float64)
    u = np.array([[T, *tau]], dtype=np.float64)
    return prob, x0, u, np.array([K], dtype=np.int32)


def test_effort_cost_and_gradient_closed_form(oracle_mod):
    prob = scenes.quad_scene(0, clutter=-1)
    rng = np.random.default_rng(5)
    S = 4
    K = rng.integers(10, 61, S).astype(np.int32)
    u = np.column_stack([MG + rng.uniform(-2, 2, S), rng.uniform(-0.02, 0.02, (S, 3))])
    x0 = np.array(prob.start, dtype=np.float64)
    spec = _spec(w_obs=0.0, w_goal=0.0, w_effort=0.7)
    J, g = oracle_mod.refine_grad(prob, spec, x0, u, K, obstacles=np.zeros((0, 6)))
    tm = TAU_MAX
    dur = K * prob.h
    e = ((u[:, 0] - MG) / MG) ** 2 + ((u[:, 1:] / tm) ** 2).sum(1)
    assert abs(J - float((dur * (1 + 0.7 * e)).sum())) < 1e-12
    g_ref = np.column_stack([dur * 0.7 * 2 * (u[:, 0] - MG) / MG ** 2, (dur * 0.7 * 2)[:, None] * u[:, 1:] / tm ** 2])
    assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-15)


def test_thrust_gradient_at_hover_closed_form(oracle_mod):
    """Level attitude at rest: z_N = z0 + (T/m - g) t^2 / 2 with t = K h,
    exact under RK4; the goal pull on z gives dJ/dT in closed form."""
    K, T = 40, MG + 1.3
    prob, x0, u, Ks = _hover_case(K, T)
    goal = [x0[0], x0[1], 0.9]
    spec = _spec(w_obs=0.0, w_goal=3.0, goal=goal, w_effort=0.0)
    J, g = oracle_mod.refine_grad(prob, spec, x0, u, Ks, obstacles=np.zeros((0, 6)))
    t = K * prob.h
    zN = x0[2] + (T / MASS - G) * t * t / 2
    assert abs(J - (t + 3.0 * (zN - 0.9) ** 2)) < 1e-10
    dT = 3.0 * 2 * (zN - 0.9) * t * t / (2 * MASS)
    assert abs(g[0, 0] - dT) < 1e-9 * max(1.0, abs(dT))
    # at level attitude with zero rates, no torque moves z: their goal gradients vanish
    assert np.all(np.abs(g[0, 1:]) < 1e-9)


def _cluttered_case(seed, S=5):
    prob = scenes.quad_scene(0, clutter=-1)
    rng = np.random.default_rng(seed)
    K = rng.integers(10, 40, S).astype(np.int32)
    u = np.column_stack([MG + rng.uniform(-1.5, 1.5, S), rng.uniform(-0.015, 0.015, (S, 3))])
    x0 = np.array(prob.start, dtype=np.float64)
    x0[6] = 0.8  # flying along +x so the path meets the boxes
    # boxes near the path: within a few margins of the straight flight line
    obs = []
    for _ in range(6):
        c = np.array([rng.uniform(0.08, 0.4), 0.5 + rng.uniform(-0.03, 0.03), 0.5 + rng.uniform(-0.03, 0.03)])
        e = rng.uniform(0.005, 0.02, 3)
        c[1] += np.sign(rng.uniform(-1, 1)) * (0.02 + e[1])
        obs.append(np.concatenate([c - e, c + e]))
    return prob, x0, u, K, np.array(obs)


def test_gradient_matches_central_differences(oracle_mod):
    for seed in range(4):
        prob, x0, u, K, obs = _cluttered_case(seed)
        if seed == 3:
            # anisotropic inertia and spinning start: the gyroscopic terms are live
            prob.param = [prob.param[0], prob.param[1], 0.01, 0.015, 0.022] + list(prob.param[5:])
            x0[9:12] = [0.8, -0.5, 0.6]
        spec = _spec()
        J, g = oracle_mod.refine_grad(prob, spec, x0, u, K, obstacles=obs)
        assert abs(J - oracle_mod.refine_cost(prob, spec, x0, u, K, obstacles=obs)) <= 1e-12 * abs(J)
        eps = 1e-6
        fd = np.zeros_like(u)
        for i in range(u.shape[0]):
            for j in range(4):
                up, um = u.copy(), u.copy()
                up[i, j] += eps
                um[i, j] -= eps
                fd[i, j] = (oracle_mod.refine_cost(prob, spec, x0, up, K, obstacles=obs)
                            - oracle_mod.refine_cost(prob, spec, x0, um, K, obstacles=obs)) / (2 * eps)
        scale = np.abs(fd).max()
        assert scale > 1e-3
        assert np.abs(g - fd).max() <= 1e-6 * scale, (seed, np.abs(g - fd).max(), scale)
        # the obstacle term matters here: dropping it changes the gradient
        _, g0 = oracle_mod.refine_grad(prob, _spec(w_obs=0.0), x0, u, K, obstacles=obs)
        assert np.abs(g - g0).max() > 1e-3 * scale


def test_penalty_value_by_hand(oracle_mod):
    """One step, one box: J = effort + w_obs sp(margin - d(p_1)) + goal."""
    prob, x0, u, K = _hover_case(1, MG)
    box = np.array([[x0[0] + 0.02, x0[1] - 0.01, x0[2] - 0.01, x0[0] + 0.03, x0[1] + 0.01, x0[2] + 0.01]])
    spec = _spec(w_obs=2.0, w_goal=0.0, w_effort=0.0, beta=100.0, margin=0.01)
    J = oracle_mod.refine_cost(prob, spec, x0, u, K, obstacles=box)
    d = 0.02  # hovering in place, 0.02 in front of the box's near face
    z = 0.01 - d
    sp = math.log1p(math.exp(100.0 * z)) / 100.0
    assert abs(J - (prob.h + 2.0 * sp)) < 1e-12


def test_validate_controls(oracle_mod):
    prob = scenes.quad_scene(0, clutter=-1)
    x0 = np.array(prob.start, dtype=np.float64)
    x0[:3] = prob.goal_c
    hover = np.array([[MG, 0, 0, 0]] * 3, np.float32)
    K = np.array([20, 20, 20], np.int32)
    r = oracle_mod.validate_controls(prob, x0, hover, K)
    assert r["valid"] and r["goal_dist"] < 1e-6
    assert abs(r["cost"] - 60 * prob.h) < 1e-12
    climb = np.array([[MG + 4, 0, 0, 0]] * 3, np.float32)  # leaves the goal ball upwards
    r = oracle_mod.validate_controls(prob, x0, climb, K)
    assert not r["valid"] and r["goal_dist"] > prob.goal_r
    # hovering inside an obstacle: in the goal, but every point collides
    boxed = scenes.quad_scene(0, clutter=-1)
    boxed.obstacles = np.array([[0.9, 0.45, 0.45, 1.0, 0.55, 0.55]], np.float32)
    r = oracle_mod.validate_controls(boxed, x0, hover, K)
    assert not r["valid"] and r["goal_dist"] < 1e-6 and r["min_clearance"] < 0
