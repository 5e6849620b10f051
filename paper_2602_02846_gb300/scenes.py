"""Seeded synthetic planning problems (inputs only, no planner arithmetic).

This module builds the problem descriptions that both the CUDA planner and the
FP64 oracle consume: dynamics limits, workspace, obstacle boxes, start state,
goal ball, cost kind, region grid and planner hyperparameters.  It holds none
of the method's arithmetic (no integration, no sampling of controls, no region
mapping, no cost evaluation); it only draws obstacle geometry from a seeded
NumPy generator and states constants.

Every numeric field is rounded to an FP32 value so that both sides of a parity
check see bit-identical inputs (the oracle widens them exactly to FP64).

The paper's four 3D environments (Forest, Narrow, House, Zig-Zag; Sec. V,
environment figure) are not available, so three synthetic scene families stand
in for them, shaped like the paper's workloads:

* ``di_scene``      -- 6D double integrator in [0,1]^3 with 20 random boxes
                       (edges U[0.05,0.15]); Euler, h=0.01; 8^3 x 2^3 regions.
* ``dubins_scene``  -- 6D Dubins airplane in a forest of 300 vertical square
                       columns (half-width U[0.01,0.03]); RK4, h=0.02;
                       16^3 x 4 regions (yaw wrapped).
* ``quad_scene``    -- 12D quadcopter in a building of 9 zig-zag walls with
                       0.04 x 0.04 openings plus 964 clutter boxes (1,000 boxes
                       total); RK4, h=0.005; 16^3 x 4^3 regions.

The dynamics themselves (Sec. V names them, without equations) are fixed by
the planner and the oracle; this module only chooses their parameters.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# Dynamics kinds, integrators and cost kinds (shared integer codes).
DI6, DUBINS6, QUAD12 = 0, 1, 2
EULER, RK4 = 0, 1
COST_PATH_LENGTH, COST_DURATION, COST_EFFORT_DURATION = 0, 1, 2

STATE_DIM = {DI6: 6, DUBINS6: 6, QUAD12: 12}
CONTROL_DIM = {DI6: 3, DUBINS6: 3, QUAD12: 4}

F32_INF = float(np.float32(np.inf))


def f32(v) -> float:
    """Round a Python number to the nearest FP32 value (returned as float)."""
    return float(np.float32(v))


@dataclasses.dataclass
class RegionAxis:
    """One axis of the region grid: state component, bin count, range, wrap."""
    state_dim: int
    bins: int
    lo: float
    hi: float
    wrap: bool = False


@dataclasses.dataclass
class Problem:
    """A complete planning query plus planner hyperparameters.

    Field meaning follows the paper's problem statement (Sec. III): dynamics
    x' = f(x,u) with compact control box U (u_lo, u_hi), state constraints
    (x_lo, x_hi) that together with the workspace box and obstacles define
    X_valid, a start state in X_valid, a goal set (a closed ball on position),
    and an additive cost.  Planner hyperparameters are the region grid (the
    decomposition R of Sec. IV), the tree capacity t_e, the branching factor
    lambda (0 = adaptive, lambda = floor(t_e/|V_A|)), I_max and the seed.
    """
    name: str
    dyn: int
    integ: int
    h: float
    k_min: int
    k_max: int
    u_lo: List[float]
    u_hi: List[float]
    x_lo: List[float]
    x_hi: List[float]
    param: List[float]
    ws_lo: List[float]
    ws_hi: List[float]
    obstacles: np.ndarray            # float32 [M, 6]: lo xyz, hi xyz
    start: np.ndarray                # float32 [n]
    goal_c: List[float]
    goal_r: float
    cost_kind: int
    w_effort: float
    axes: List[RegionAxis]
    tree_cap: int
    lam: int
    i_max: int = 10
    seed: int = 0
    iterations: int = 200
    region_capacity: int = 0         # regions the planner's workspace holds (0: this grid's count)

    @property
    def n(self) -> int:
        return STATE_DIM[self.dyn]

    @property
    def m(self) -> int:
        return CONTROL_DIM[self.dyn]

    @property
    def n_regions(self) -> int:
        r = 1
        for a in self.axes:
            r *= a.bins
        return r

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _f32_list(v) -> List[float]:
    return [f32(x) for x in v]


def _pad(v, k, fill):
    v = list(v)
    return v + [fill] * (k - len(v))


def _box_point_dist(box: np.ndarray, p: np.ndarray) -> float:
    """Euclidean distance from point p to a closed axis-aligned box."""
    d = np.maximum(np.maximum(box[:3] - p, p - box[3:]), 0.0)
    return float(np.sqrt((d * d).sum()))


def _finish_problem(**kw) -> Problem:
    kw["h"] = f32(kw["h"])
    for key in ("u_lo", "u_hi", "x_lo", "x_hi", "param", "ws_lo", "ws_hi", "goal_c"):
        kw[key] = _f32_list(kw[key])
    kw["goal_r"] = f32(kw["goal_r"])
    kw["w_effort"] = f32(kw["w_effort"])
    kw["obstacles"] = np.ascontiguousarray(np.asarray(kw["obstacles"], dtype=np.float32).reshape(-1, 6))
    kw["start"] = np.ascontiguousarray(np.asarray(kw["start"], dtype=np.float32))
    kw["axes"] = [RegionAxis(a.state_dim, a.bins, f32(a.lo), f32(a.hi), a.wrap) for a in kw["axes"]]
    return Problem(**kw)


# --------------------------------------------------------------------------
# 6D double integrator (state p, v; control a)
# --------------------------------------------------------------------------
def di_obstacles(seed: int, count: int = 20, edge=(0.05, 0.15),
                 start=(0.05, 0.05, 0.05), goal=(0.95, 0.95, 0.95), goal_r=0.05,
                 clearance=0.05) -> np.ndarray:
    """Random boxes: centres U[0,1]^3, per-axis edges U[edge], clipped to the
    unit workspace; boxes closer than ``clearance`` to the start point or to
    the goal ball are redrawn."""
    rng = np.random.default_rng([0x5CE7E, 1, seed])
    s = np.asarray(start, dtype=np.float64)
    g = np.asarray(goal, dtype=np.float64)
    out = []
    while len(out) < count:
        c = rng.uniform(0.0, 1.0, 3)
        e = rng.uniform(edge[0], edge[1], 3)
        box = np.concatenate([np.clip(c - e / 2, 0, 1), np.clip(c + e / 2, 0, 1)])
        box = box.astype(np.float32).astype(np.float64)
        if _box_point_dist(box, s) <= clearance:
            continue
        if _box_point_dist(box, g) <= goal_r + clearance:
            continue
        out.append(box)
    return np.asarray(out, dtype=np.float32).reshape(-1, 6)


def di_scene(seed: int = 0, n_obstacles: int = 20, tree_cap: int = 32768, lam: int = 16,
             grid_pos: int = 8, grid_vel: int = 2, planner_seed: Optional[int] = None,
             iterations: int = 200, i_max: int = 10) -> Problem:
    """6D double integrator: p' = v, v' = a, |a_i| <= 1, |v_i| <= 1, Euler
    h = 0.01 with 5..30 steps (0.05-0.30 s), cost = path length."""
    start = [0.05, 0.05, 0.05, 0.0, 0.0, 0.0]
    goal = [0.95, 0.95, 0.95]
    obs = di_obstacles(seed, n_obstacles) if n_obstacles > 0 else np.zeros((0, 6), np.float32)
    inf = F32_INF
    axes = [RegionAxis(d, grid_pos, 0.0, 1.0) for d in range(3)] + \
           [RegionAxis(3 + d, grid_vel, -1.0, 1.0) for d in range(3)]
    return _finish_problem(
        name="di6", dyn=DI6, integ=EULER, h=0.01, k_min=5, k_max=30,
        u_lo=[-1, -1, -1], u_hi=[1, 1, 1],
        x_lo=[-inf, -inf, -inf, -1, -1, -1], x_hi=[inf, inf, inf, 1, 1, 1],
        param=[0.0] * 8, ws_lo=[0, 0, 0], ws_hi=[1, 1, 1],
        obstacles=obs, start=start, goal_c=goal, goal_r=0.05,
        cost_kind=COST_PATH_LENGTH, w_effort=0.0, axes=axes,
        tree_cap=tree_cap, lam=lam, i_max=i_max,
        seed=seed if planner_seed is None else planner_seed, iterations=iterations)


# --------------------------------------------------------------------------
# 6D Dubins airplane (x, y, z, yaw, pitch, speed; controls yaw rate, pitch rate, accel)
# --------------------------------------------------------------------------
def dubins_obstacles(seed: int, count: int = 300, half=(0.01, 0.03),
                     start=(0.05, 0.05), goal=(0.95, 0.95), clearance=0.1) -> np.ndarray:
    """Vertical square columns spanning z in [0,1]: centres U[0,1]^2,
    half-width U[half]; columns within ``clearance`` (xy) of the start or the
    goal centre are redrawn."""
    rng = np.random.default_rng([0x5CE7E, 2, seed])
    s = np.asarray(start, dtype=np.float64)
    g = np.asarray(goal, dtype=np.float64)
    out = []
    while len(out) < count:
        c = rng.uniform(0.0, 1.0, 2)
        r = rng.uniform(half[0], half[1])
        lo = np.clip(c - r, 0, 1)
        hi = np.clip(c + r, 0, 1)
        box2 = np.concatenate([lo, hi]).astype(np.float32).astype(np.float64)

        def dist2(p):
            d = np.maximum(np.maximum(box2[:2] - p, p - box2[2:]), 0.0)
            return float(np.sqrt((d * d).sum()))
        if dist2(s) <= clearance or dist2(g) <= clearance:
            continue
        out.append([box2[0], box2[1], 0.0, box2[2], box2[3], 1.0])
    return np.asarray(out, dtype=np.float32).reshape(-1, 6)


def dubins_scene(seed: int = 0, n_obstacles: int = 300, tree_cap: int = 1 << 20, lam: int = 64,
                 grid_pos: int = 16, grid_yaw: int = 4, planner_seed: Optional[int] = None,
                 iterations: int = 200, i_max: int = 10) -> Problem:
    """6D Dubins airplane: x' = v cos(psi) cos(gamma), y' = v sin(psi) cos(gamma),
    z' = v sin(gamma), psi' = u0, gamma' = u1, v' = u2; |u0|,|u1| <= 0.5,
    |u2| <= 0.3; v in [0.1, 0.3], |gamma| <= pi/4; RK4 h = 0.02 with 5..25
    steps; cost = duration."""
    start = [0.05, 0.05, 0.5, math.pi / 4, 0.0, 0.2]
    goal = [0.95, 0.95, 0.5]
    obs = dubins_obstacles(seed, n_obstacles) if n_obstacles > 0 else np.zeros((0, 6), np.float32)
    inf = F32_INF
    q = math.pi / 4
    axes = [RegionAxis(d, grid_pos, 0.0, 1.0) for d in range(3)] + \
           [RegionAxis(3, grid_yaw, -math.pi, math.pi, wrap=True)]
    return _finish_problem(
        name="dubins6", dyn=DUBINS6, integ=RK4, h=0.02, k_min=5, k_max=25,
        u_lo=[-0.5, -0.5, -0.3], u_hi=[0.5, 0.5, 0.3],
        x_lo=[-inf, -inf, -inf, -inf, -q, 0.1], x_hi=[inf, inf, inf, inf, q, 0.3],
        param=[0.0] * 8, ws_lo=[0, 0, 0], ws_hi=[1, 1, 1],
        obstacles=obs, start=start, goal_c=goal, goal_r=0.05,
        cost_kind=COST_DURATION, w_effort=0.0, axes=axes,
        tree_cap=tree_cap, lam=lam, i_max=i_max,
        seed=seed if planner_seed is None else planner_seed, iterations=iterations)


# --------------------------------------------------------------------------
# 12D quadcopter (p, roll/pitch/yaw ZYX, v, body rates; controls thrust + torques)
# --------------------------------------------------------------------------
QUAD_MASS, QUAD_G, QUAD_J = 1.0, 9.81, 0.01
QUAD_T_DEV, QUAD_TAU_MAX = 4.0, 0.02


def _wall_boxes(x: float, cy: float, cz: float, half_open=0.02, thick=0.01):
    """Four boxes forming a wall at x with a square opening centred (cy, cz)."""
    x0, x1 = x - thick / 2, x + thick / 2
    y0, y1 = cy - half_open, cy + half_open
    z0, z1 = cz - half_open, cz + half_open
    return [
        [x0, 0.0, 0.0, x1, y0, 1.0],
        [x0, y1, 0.0, x1, 1.0, 1.0],
        [x0, y0, 0.0, x1, y1, z0],
        [x0, y0, z1, x1, y1, 1.0],
    ]


def quad_openings():
    """Opening centres (y, z) of the nine walls, alternating between two corners."""
    return [(0.3, 0.3) if i % 2 == 0 else (0.7, 0.7) for i in range(9)]


def _seg_box_dist(box, a, b, samples=9):
    return min(_box_point_dist(box, a + (b - a) * t) for t in np.linspace(0.0, 1.0, samples))


def _near_any_segment(box, seg_points, limit):
    """True if any sample point of the opening axes lies within ``limit`` of
    the box (same test as _seg_box_dist over every segment, vectorised)."""
    d = np.maximum(np.maximum(box[:3] - seg_points, seg_points - box[3:]), 0.0)
    return bool((np.sqrt((d * d).sum(axis=1)) <= limit).any())


def voxel_connected(obstacles: np.ndarray, start, goal, ws_lo=(0, 0, 0), ws_hi=(1, 1, 1),
                    res: float = 0.005) -> bool:
    """Certify point-robot connectivity from start to goal on a voxel grid.

    A voxel is blocked when its closed cell touches any closed box; start and
    goal must lie in the same 6-connected free component.
    """
    from scipy import ndimage
    n = [int(round((hi - lo) / res)) for lo, hi in zip(ws_lo, ws_hi)]
    free = np.ones(n, dtype=bool)
    for b in np.asarray(obstacles, dtype=np.float64):
        i0 = [max(0, int(math.floor((b[a] - ws_lo[a]) / res)) - 1) for a in range(3)]
        i1 = [min(n[a], int(math.ceil((b[3 + a] - ws_lo[a]) / res)) + 1) for a in range(3)]
        free[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] = False
    lab, _ = ndimage.label(free)
    si = tuple(min(n[a] - 1, int((start[a] - ws_lo[a]) / res)) for a in range(3))
    gi = tuple(min(n[a] - 1, int((goal[a] - ws_lo[a]) / res)) for a in range(3))
    return bool(lab[si] != 0 and lab[si] == lab[gi])


def quad_obstacles(seed: int, clutter: int = 964, edge=(0.01, 0.03), certify: bool = True,
                   start=(0.05, 0.5, 0.5), goal=(0.95, 0.5, 0.5), walls: bool = True) -> np.ndarray:
    """Building world: 9 walls at x = 0.1 i (36 boxes) with 0.04 x 0.04
    openings in alternating corners, plus ``clutter`` random boxes kept 0.04
    away from each opening axis and 0.08 away from start and goal.  The scene
    is redrawn (next sub-seed) until a 0.005 voxel BFS connects start to goal.
    walls=False keeps only the clutter (an open cluttered room)."""
    attempt = 0
    while True:
        rng = np.random.default_rng([0x5CE7E, 3, seed, attempt])
        boxes = []
        axes = []
        for i, (cy, cz) in enumerate(quad_openings()):
            x = 0.1 * (i + 1)
            if walls:
                boxes += _wall_boxes(x, cy, cz)
            axes.append((np.array([x - 0.05, cy, cz]), np.array([x + 0.05, cy, cz])))
        s = np.asarray(start, dtype=np.float64)
        g = np.asarray(goal, dtype=np.float64)
        ts = np.linspace(0.0, 1.0, 9)[:, None]
        seg_points = np.concatenate([a + (b - a) * ts for a, b in axes])
        n_clutter = 0
        while n_clutter < clutter:
            c = rng.uniform(0.0, 1.0, 3)
            e = rng.uniform(edge[0], edge[1], 3)
            box = np.concatenate([np.clip(c - e / 2, 0, 1), np.clip(c + e / 2, 0, 1)])
            box = box.astype(np.float32).astype(np.float64)
            if _box_point_dist(box, s) <= 0.08 or _box_point_dist(box, g) <= 0.08:
                continue
            if _near_any_segment(box, seg_points, 0.04):
                continue
            boxes.append(list(box))
            n_clutter += 1
        arr = np.asarray(boxes, dtype=np.float32).reshape(-1, 6)
        if not certify or voxel_connected(arr, start, goal):
            return arr
        attempt += 1


def quad_scene(seed: int = 0, clutter: int = 964, tree_cap: int = 1 << 22, lam: int = 128,
               grid_pos: int = 16, grid_vel: int = 4, planner_seed: Optional[int] = None,
               iterations: int = 200, i_max: int = 10, certify: bool = True, walls: bool = True) -> Problem:
    """12D quadcopter, state (p, phi/theta/psi ZYX, v, omega), control
    (thrust T, torques tau): p' = v, v' = (T/m) R e3 - g e3,
    (phi,theta,psi)' = W(phi,theta) omega, omega' = J^-1 (tau - omega x J omega);
    m = 1, J = diag(0.01), g = 9.81; T in [mg-4, mg+4], |tau_i| <= 0.02;
    |v_i| <= 1, |phi|,|theta| <= pi/4, |omega_i| <= 2; RK4 h = 0.005 with
    10..60 steps; cost = duration x (1 + w e(u)), e(u) = ((T-mg)/mg)^2 +
    sum (tau_i/tau_max)^2, w = 1."""
    start = [0.05, 0.5, 0.5] + [0.0] * 9
    goal = [0.95, 0.5, 0.5]
    obs = quad_obstacles(seed, clutter, certify=certify, walls=walls) if clutter >= 0 else np.zeros((0, 6), np.float32)
    inf = F32_INF
    q = math.pi / 4
    mg = QUAD_MASS * QUAD_G
    axes = [RegionAxis(d, grid_pos, 0.0, 1.0) for d in range(3)] + \
           [RegionAxis(6 + d, grid_vel, -1.0, 1.0) for d in range(3)]
    tm = QUAD_TAU_MAX
    return _finish_problem(
        name="quad12", dyn=QUAD12, integ=RK4, h=0.005, k_min=10, k_max=60,
        u_lo=[mg - QUAD_T_DEV, -tm, -tm, -tm], u_hi=[mg + QUAD_T_DEV, tm, tm, tm],
        x_lo=[-inf, -inf, -inf, -q, -q, -inf, -1, -1, -1, -2, -2, -2],
        x_hi=[inf, inf, inf, q, q, inf, 1, 1, 1, 2, 2, 2],
        param=[QUAD_MASS, QUAD_G, QUAD_J, QUAD_J, QUAD_J, tm, 0.0, 0.0],
        ws_lo=[0, 0, 0], ws_hi=[1, 1, 1],
        obstacles=obs, start=start, goal_c=goal, goal_r=0.05,
        cost_kind=COST_EFFORT_DURATION, w_effort=1.0, axes=axes,
        tree_cap=tree_cap, lam=lam, i_max=i_max,
        seed=seed if planner_seed is None else planner_seed, iterations=iterations)


def scene(kind: str, seed: int = 0, **kw) -> Problem:
    """Build a scene by family name: 'di', 'dubins' or 'quad'."""
    return {"di": di_scene, "dubins": dubins_scene, "quad": quad_scene}[kind](seed=seed, **kw)


def obstacle_volume_fraction(obstacles: np.ndarray, res: float = 0.005) -> float:
    """Fraction of the unit workspace covered by the union of the boxes."""
    n = int(round(1.0 / res))
    occ = np.zeros((n, n, n), dtype=bool)
    for b in np.asarray(obstacles, dtype=np.float64):
        i0 = [max(0, int(round(b[a] / res))) for a in range(3)]
        i1 = [min(n, int(round(b[3 + a] / res))) for a in range(3)]
        occ[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] = True
    return float(occ.mean())


def mixed_problem(rng: np.random.Generator, kind: int, iterations: int = 100) -> Problem:
    """One problem of the batched / served mix: family ``kind`` (0 double
    integrator on the 16^3 x 2^3 grid, 1 Dubins airplane, 2 quadcopter),
    10-1,000 seeded boxes (walls plus clutter for the quadcopter), tree
    capacity 2^14..2^20 (log-uniform), the family's region grid and lambda.
    Quadcopter buildings are not voxel-certified here (generation time)."""
    n_obs = int(rng.integers(10, 1001))
    cap = 1 << int(rng.integers(14, 21))
    s = int(rng.integers(1 << 30))
    if kind == 0:
        return di_scene(s, n_obstacles=n_obs, tree_cap=cap, grid_pos=16, iterations=iterations)
    if kind == 1:
        return dubins_scene(s, n_obstacles=n_obs, tree_cap=cap, iterations=iterations)
    return quad_scene(s, clutter=max(0, n_obs - 36), tree_cap=cap, certify=False, iterations=iterations)


def mixed_batch(count: int = 512, seed: int = 0, iterations: int = 100) -> List[Problem]:
    """Independent problems of uneven size for batched planning: the three
    families in turn, each drawn by mixed_problem."""
    rng = np.random.default_rng([0x5CE7E, 9, seed])
    return [mixed_problem(rng, k % 3, iterations) for k in range(count)]


def poisson_requests(rate: float, duration: float, seed: int = 0, iterations: int = 100):
    """A request stream for the serving loop: Poisson arrivals at ``rate``
    per second over ``duration`` seconds, each a mixed_problem of a family
    drawn uniformly.  Returns [(arrival_seconds, Problem)] in arrival order."""
    rng = np.random.default_rng([0x5E27E, 11, seed])
    out, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            return out
        out.append((t, mixed_problem(rng, int(rng.integers(3)), iterations)))


def refine_batch(count: int = 4096, seed: int = 0, segments=(64, 512), steps=(10, 60), n_obstacles: int = 1000):
    """Control sequences of the refinement workload for the 12D quadcopter:
    ``count`` trajectories from the quadcopter start state, each with a
    segment count drawn from ``segments`` and per-segment step counts from
    ``steps`` (both inclusive), thrust mg + U(-0.5, 0.5) and torques
    U(-0.001, 0.001) held per segment, among the 1,000-box building
    (``n_obstacles`` boxes of it).  Returns dict(problem, x0, u, steps, n_seg,
    obstacles); rows past a trajectory's segment count are zero."""
    prob = quad_scene(seed, certify=False)
    rng = np.random.default_rng([0x2EF1E, 5, seed])
    S = int(segments[1])
    n_seg = rng.integers(segments[0], segments[1] + 1, count).astype(np.int32)
    st = rng.integers(steps[0], steps[1] + 1, (count, S)).astype(np.int32)
    mg = float(np.float32(QUAD_MASS * QUAD_G))
    u = np.zeros((count, S, 4), np.float32)
    u[:, :, 0] = mg + rng.uniform(-0.5, 0.5, (count, S))
    u[:, :, 1:] = rng.uniform(-0.001, 0.001, (count, S, 3))
    mask = np.arange(S)[None, :] < n_seg[:, None]
    u *= mask[:, :, None]
    st *= mask
    x0 = np.tile(np.asarray(prob.start, np.float32), (count, 1))
    obs = np.asarray(prob.obstacles, np.float32)[:n_obstacles]
    return dict(problem=prob, x0=x0, u=u, steps=st, n_seg=n_seg, obstacles=obs)

