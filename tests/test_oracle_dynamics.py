"""Oracle pins: dynamics, integrators and edge costs (PropagateODE of Alg. 2).

Pins are closed forms and hand-derived values, never the oracle's own code:
Euler on the double integrator, RK4 exactness on polynomials of degree <= 4,
quadcopter free fall / hover / constant roll torque, hand-evaluated rotation
and Euler-rate matrices, Dubins straight and circular flight with the
integrator's convergence order, and the three edge-cost definitions.
"""
import math

import numpy as np
import pytest

from paper_2602_02846_gb300 import scenes


def di(**kw):
    return scenes.di_scene(0, n_obstacles=0, **kw)


def dubins(**kw):
    return scenes.dubins_scene(0, n_obstacles=0, **kw)


def quad(**kw):
    return scenes.quad_scene(0, clutter=0, certify=False, **kw)


def test_di_euler_closed_form(oracle_mod):
    """p_K = p0 + K h v0 + h^2 a K(K-1)/2, v_K = v0 + K h a (forward Euler)."""
    p = di()
    h = float(np.float32(0.01))
    x0 = np.array([0.3, 0.4, 0.5, 0.1, -0.2, 0.05])
    a = np.array([0.5, -0.25, 0.125], dtype=np.float32)
    for K in (1, 7, 30):
        r = oracle_mod.rollout(p, x0, a, K)
        ad = a.astype(np.float64)
        pk = x0[:3] + K * h * x0[3:] + h * h * ad * K * (K - 1) / 2
        vk = x0[3:] + K * h * ad
        np.testing.assert_allclose(r["x_end"][:3], pk, rtol=0, atol=1e-14)
        np.testing.assert_allclose(r["x_end"][3:], vk, rtol=0, atol=1e-14)


def test_di_rk4_exact_for_quadratic(oracle_mod):
    p = di().replace(integ=scenes.RK4)
    h = float(np.float32(0.01))
    x0 = np.array([0.2, 0.2, 0.2, 0.3, 0.0, -0.1])
    a = np.array([1.0, -1.0, 0.5], dtype=np.float32)
    K = 17
    t = K * h
    r = oracle_mod.rollout(p, x0, a, K)
    ad = a.astype(np.float64)
    np.testing.assert_allclose(r["x_end"][:3], x0[:3] + x0[3:] * t + 0.5 * ad * t * t, atol=1e-14)
    np.testing.assert_allclose(r["x_end"][3:], x0[3:] + ad * t, atol=1e-14)


def test_quad_free_fall_and_hover(oracle_mod):
    p = quad()
    h = float(np.float32(0.005))
    g = float(np.float32(9.81))
    x0 = np.zeros(12)
    x0[:3] = [0.5, 0.5, 0.9]
    # thrust 0: z = z0 - g t^2 / 2 (RK4 exact), no lateral motion
    xn = x0.copy()
    u = np.array([0.0, 0.0, 0.0, 0.0])
    for _ in range(20):
        xn = oracle_mod.step(p, xn, u)
    t = 20 * h
    assert abs(xn[2] - (0.9 - 0.5 * g * t * t)) < 1e-14
    assert abs(xn[8] + g * t) < 1e-13
    assert np.all(xn[:2] == 0.5)
    assert np.all(np.abs(xn[[3, 4, 5, 6, 7, 9, 10, 11]]) < 1e-15)
    # hover: T = m g, level, at rest -> derivative exactly zero
    m = float(np.float32(1.0))
    dx = oracle_mod.deriv(p, x0, np.array([m * g, 0, 0, 0]))
    assert np.all(dx == 0.0)


def test_quad_constant_roll_torque(oracle_mod):
    """Level at rest with tau_x: phi = tau/(2 Jx) t^2, p = tau/Jx t (RK4 exact)."""
    p = quad()
    h = float(np.float32(0.005))
    J = float(np.float32(0.01))
    tau = 0.01
    x = np.zeros(12)
    x[:3] = [0.5, 0.5, 0.5]
    u = np.array([0.0, tau, 0.0, 0.0])
    for _ in range(8):
        x = oracle_mod.step(p, x, u)
    t = 8 * h
    assert abs(x[9] - tau / J * t) < 1e-14
    # theta stays 0, so W's first row gives phi' = p exactly
    assert abs(x[3] - 0.5 * tau / J * t * t) < 1e-14
    assert abs(x[4]) < 1e-15 and abs(x[5]) < 1e-15


def test_quad_rotation_column_hand_values(oracle_mod):
    """v' = (T/m) R e3 - g e3 with R = Rz(psi) Ry(theta) Rx(phi)."""
    p = quad()
    g = float(np.float32(9.81))
    T = 10.0

    def acc(phi, th, psi):
        x = np.zeros(12)
        x[3:6] = [phi, th, psi]
        return oracle_mod.deriv(p, x, np.array([T, 0, 0, 0]))[6:9]
    th = 0.3
    np.testing.assert_allclose(acc(0, th, 0), [T * math.sin(th), 0, T * math.cos(th) - g], atol=1e-14)
    ph = 0.2
    np.testing.assert_allclose(acc(ph, 0, 0), [0, -T * math.sin(ph), T * math.cos(ph) - g], atol=1e-14)
    # yaw pi/2 turns the pitch tilt from +x into +y
    np.testing.assert_allclose(acc(0, th, math.pi / 2), [0, T * math.sin(th), T * math.cos(th) - g], atol=1e-14)
    # roll and pitch together (Rx applied first): R e3 = (s_th c_ph, -s_ph, c_th c_ph) at psi = 0
    np.testing.assert_allclose(acc(ph, th, 0), [T * math.sin(th) * math.cos(ph), -T * math.sin(ph),
                                               T * math.cos(th) * math.cos(ph) - g], atol=1e-14)
    # general angles: third column of the matrix product Rz(psi) @ Ry(theta) @ Rx(phi)
    ph, th, ps = 0.3, -0.2, 1.1
    c, s = math.cos, math.sin
    Rx = np.array([[1, 0, 0], [0, c(ph), -s(ph)], [0, s(ph), c(ph)]])
    Ry = np.array([[c(th), 0, s(th)], [0, 1, 0], [-s(th), 0, c(th)]])
    Rz = np.array([[c(ps), -s(ps), 0], [s(ps), c(ps), 0], [0, 0, 1]])
    e3 = (Rz @ Ry @ Rx)[:, 2]
    np.testing.assert_allclose(acc(ph, th, ps), T * e3 - np.array([0, 0, g]), atol=1e-13)


def test_quad_euler_rates_hand_values(oracle_mod):
    """(phi,theta,psi)' = W(phi,theta) omega, hand-evaluated at phi = pi/2 and at phi = 0."""
    p = quad()
    x = np.zeros(12)
    th = 0.4
    x[3:6] = [math.pi / 2, th, 0.0]
    x[9:12] = [0.1, 0.2, 0.3]
    d = oracle_mod.deriv(p, x, np.array([0.0, 0, 0, 0]))
    # W(pi/2, th) = [[1, t, 0], [0, 0, -1], [0, 1/c, 0]]
    t, c = math.tan(th), math.cos(th)
    np.testing.assert_allclose(d[3:6], [0.1 + t * 0.2, -0.3, 0.2 / c], atol=1e-14)
    x[3] = 0.0
    d = oracle_mod.deriv(p, x, np.array([0.0, 0, 0, 0]))
    # W(0, th) = [[1, 0, t], [0, 1, 0], [0, 0, 1/c]]
    np.testing.assert_allclose(d[3:6], [0.1 + t * 0.3, 0.2, 0.3 / c], atol=1e-14)


def test_quad_gyroscopic_term(oracle_mod):
    """omega' = J^-1 (tau - omega x J omega) with unequal inertia."""
    p = quad().replace(param=[1.0, 9.81, 0.01, 0.02, 0.03, 0.02, 0.0, 0.0])
    x = np.zeros(12)
    w = np.array([0.5, -0.4, 0.3])
    x[9:12] = w
    tau = np.array([0.001, 0.002, -0.003])
    d = oracle_mod.deriv(p, x, np.concatenate([[9.81], tau]))
    J = np.array(p.param[2:5], dtype=np.float64)
    Jw = J * w
    expect = (tau - np.cross(w, Jw)) / J
    np.testing.assert_allclose(d[9:12], expect, rtol=1e-14, atol=1e-14)


def test_dubins_straight_flight(oracle_mod):
    """u = 0: a straight line at constant speed along (c_psi c_gam, s_psi c_gam, s_gam)."""
    p = dubins()
    h = float(np.float32(0.02))
    psi, gam, v = math.pi / 6, 0.1, 0.2
    x0 = np.array([0.2, 0.3, 0.4, psi, gam, v])
    K = 12
    r = oracle_mod.rollout(p, x0, np.zeros(3, np.float32), K)
    t = K * h
    d = np.array([math.cos(psi) * math.cos(gam), math.sin(psi) * math.cos(gam), math.sin(gam)])
    np.testing.assert_allclose(r["x_end"][:3], x0[:3] + v * t * d, atol=1e-14)
    np.testing.assert_allclose(r["x_end"][3:], x0[3:], atol=0)


def _circle_error(oracle_mod, integ, h):
    p = dubins().replace(integ=integ, h=h)
    v, w = 0.2, 0.5
    x = np.array([0.5, 0.5, 0.5, 0.0, 0.0, v])
    T = 1.0
    n = int(round(T / h))
    for _ in range(n):
        x = oracle_mod.step(p, x, np.array([w, 0.0, 0.0]))
    R = v / w
    # exact: x = x0 + R sin(w t), y = y0 + R (1 - cos(w t))
    ex = 0.5 + R * math.sin(w * T)
    ey = 0.5 + R * (1 - math.cos(w * T))
    return math.hypot(x[0] - ex, x[1] - ey)


def test_dubins_circle_convergence_orders(oracle_mod):
    """Constant yaw rate at gamma = 0 is a circle of radius v/omega; RK4 error
    falls ~16x per halving of h, Euler error ~2x."""
    e1 = _circle_error(oracle_mod, scenes.RK4, 0.1)
    e2 = _circle_error(oracle_mod, scenes.RK4, 0.05)
    assert e1 < 1e-6
    assert 12.0 < e1 / e2 < 20.0
    f1 = _circle_error(oracle_mod, scenes.EULER, 0.01)
    f2 = _circle_error(oracle_mod, scenes.EULER, 0.005)
    assert 1.8 < f1 / f2 < 2.2


def test_edge_costs(oracle_mod):
    # path length of a constant-velocity DI segment = K h |v|
    p = di()
    h = float(np.float32(0.01))
    x0 = np.array([0.5, 0.5, 0.5, 0.3, -0.4, 0.2])
    r = oracle_mod.rollout(p, x0, np.zeros(3, np.float32), 20)
    assert r["valid"]
    assert abs(r["edge_cost"] - 20 * h * math.sqrt(0.09 + 0.16 + 0.04)) < 1e-14
    # accelerating from rest along x: length = a t^2/2 exactly for Euler's
    # polygon?  Euler positions are h^2 a k(k-1)/2; sum of |steps| = final x - x0.
    r = oracle_mod.rollout(p, np.array([0.2, 0.5, 0.5, 0, 0, 0]), np.array([1.0, 0, 0], np.float32), 10)
    assert abs(r["edge_cost"] - (r["x_end"][0] - 0.2)) < 1e-14
    # duration
    pd = dubins()
    x0 = np.array([0.5, 0.5, 0.5, 0.0, 0.0, 0.2])
    r = oracle_mod.rollout(pd, x0, np.zeros(3, np.float32), 9)
    assert r["edge_cost"] == 9 * float(np.float32(0.02))
    # effort + duration: hover -> e = 0; full thrust deviation and torque
    pq = quad()
    hq = float(np.float32(0.005))
    mg = float(np.float32(1.0)) * float(np.float32(9.81))
    xq = np.zeros(12)
    xq[:3] = [0.5, 0.5, 0.5]
    r = oracle_mod.rollout(pq, xq, np.array([mg, 0, 0, 0], np.float32), 10)
    assert abs(r["edge_cost"] - 10 * hq * (1.0 + 0.0)) < 1e-6  # mg rounded to FP32 in u
    T = np.float32(mg + 2.0)
    tau = np.float32(0.01)
    r = oracle_mod.rollout(pq, xq, np.array([T, tau, 0, -tau], np.float32), 4)
    tmax = float(np.float32(0.02))
    e = ((float(T) - mg) / mg) ** 2 + 2 * (float(tau) / tmax) ** 2
    assert abs(r["edge_cost"] - 4 * hq * (1 + e)) < 1e-14
