"""ctypes front end of the FP64 planning oracle (plain C, single thread).

TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA planner; only
the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it.  It does not import the planner package and the planner package
does not import it; both consume the same seeded scene description (any object
with the fields of ``scenes.Problem``).

Each wrapper names the part of the paper it follows (see kpx_oracle.c).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kpx_oracle.c")
_HDR = os.path.join(_HERE, "kpx_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkpx_oracle.so")
_lock = threading.Lock()
_lib = None

KEY_INF = 0xFFFFFFFFFFFFFFFF
SET_A, SET_I, SET_T = 1, 2, 3
OK, INVALID, TREE_FULL, NO_SOLUTION = 0, 1, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("dyn", C.c_int32), ("integ", C.c_int32), ("n", C.c_int32), ("m", C.c_int32),
        ("h", C.c_double),
        ("k_min", C.c_int32), ("k_max", C.c_int32),
        ("u_lo", C.c_float * 8), ("u_hi", C.c_float * 8),
        ("x_lo", C.c_double * 16), ("x_hi", C.c_double * 16),
        ("param", C.c_double * 8),
        ("ws_lo", C.c_double * 3), ("ws_hi", C.c_double * 3),
        ("goal_c", C.c_double * 3), ("goal_r", C.c_double),
        ("cost_kind", C.c_int32), ("pad0", C.c_int32),
        ("w_effort", C.c_double),
        ("n_axes", C.c_int32), ("pad1", C.c_int32),
        ("ax_dim", C.c_int32 * 8), ("ax_bins", C.c_int32 * 8), ("ax_wrap", C.c_int32 * 8),
        ("ax_lo", C.c_float * 8), ("ax_hi", C.c_float * 8),
        ("tree_cap", C.c_int32), ("lam", C.c_int32), ("i_max", C.c_int32), ("n_obs", C.c_int32),
        ("seed", C.c_uint64),
        ("obs", C.POINTER(C.c_double)),
    ]


class View(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("R", C.c_int32), ("n", C.c_int32), ("m", C.c_int32),
        ("n_nodes", C.c_int32), ("count_A", C.c_int32), ("iter", C.c_int32), ("tree_full", C.c_int32),
        ("first_solution_iter", C.c_int32), ("last_lambda", C.c_int32),
        ("goal_key", C.c_uint64),
        ("last_candidates", C.c_int64), ("last_valid", C.c_int64), ("last_winners", C.c_int64),
        ("total_candidates", C.c_int64), ("total_valid", C.c_int64), ("total_winners", C.c_int64),
        ("x", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_float)), ("K", C.POINTER(C.c_int32)),
        ("parent", C.POINTER(C.c_int32)), ("cost", C.POINTER(C.c_double)),
        ("key", C.POINTER(C.c_uint64)), ("region", C.POINTER(C.c_int32)),
        ("set", C.POINTER(C.c_uint8)), ("icount", C.POINTER(C.c_uint8)),
        ("region_key", C.POINTER(C.c_uint64)), ("VA", C.POINTER(C.c_int32)),
    ]


def _p(arr, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


def load_library(path: str):
    """Open an oracle shared library at ``path`` with its signatures set."""
    L = C.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_LIB)
    return _lib


def _declare(L):
    """Set argument and return types of every exported oracle function."""
    vp = C.c_void_p
    L.kpo_philox4x32_10.argtypes = [vp, vp, vp]
    L.kpo_sample_control.argtypes = [C.POINTER(Problem), C.c_uint32, C.c_uint32, C.c_uint32, vp, vp]
    L.kpo_deriv.argtypes = [C.POINTER(Problem), vp, vp, vp]
    L.kpo_step.argtypes = [C.POINTER(Problem), vp, vp, vp]
    L.kpo_point_valid.argtypes = [C.POINTER(Problem), vp]
    L.kpo_point_valid.restype = C.c_int32
    L.kpo_point_margin.argtypes = [C.POINTER(Problem), vp]
    L.kpo_point_margin.restype = C.c_double
    L.kpo_point_clearance.argtypes = [C.POINTER(Problem), vp]
    L.kpo_point_clearance.restype = C.c_double
    L.kpo_rollout.argtypes = [C.POINTER(Problem), vp, vp, C.c_int32, vp, vp, vp, vp, vp]
    L.kpo_rollout.restype = C.c_int32
    L.kpo_region.argtypes = [C.POINTER(Problem), vp, vp]
    L.kpo_region.restype = C.c_int32
    L.kpo_in_goal.argtypes = [C.POINTER(Problem), vp, vp]
    L.kpo_in_goal.restype = C.c_int32
    L.kpo_pack_key.argtypes = [C.c_float, C.c_uint32]
    L.kpo_pack_key.restype = C.c_uint64
    L.kpo_propagate.argtypes = [C.POINTER(Problem), C.c_uint32, C.c_int32, vp, vp, vp, C.c_int32,
                                C.c_int64, vp] + [vp] * 11
    L.kpo_select_winners.argtypes = [C.c_int32, vp, vp, C.c_int64, vp, vp, vp, C.c_int32, C.c_int32,
                                     vp, vp, vp]
    L.kpo_select_winners.restype = C.c_int32
    L.kpo_prune.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, C.c_int32]
    L.kpo_compact.argtypes = [C.c_int32, vp, vp, vp]
    L.kpo_compact.restype = C.c_int32
    L.kpo_append.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32] + [vp] * 7 + [vp] * 11
    L.kpo_append.restype = C.c_int32
    L.kpo_create.argtypes = [C.POINTER(Problem), vp]
    L.kpo_create.restype = vp
    L.kpo_iterate.argtypes = [vp, C.c_int32]
    L.kpo_iterate.restype = C.c_int32
    L.kpo_view_state.argtypes = [vp, C.POINTER(View)]
    L.kpo_best_trajectory.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
    L.kpo_best_trajectory.restype = C.c_int32
    L.kpo_destroy.argtypes = [vp]
    L.kpo_revalidate.argtypes = [C.POINTER(Problem), C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.kpo_revalidate.restype = C.c_int32
    L.kpo_remap_regions.argtypes = [C.POINTER(Problem), C.c_int32, vp, vp, vp, vp, vp, vp, vp]
    L.kpo_box_distance.argtypes = [vp, vp, vp]
    L.kpo_box_distance.restype = C.c_double
    L.kpo_refine_cost.argtypes = [C.POINTER(Problem), C.POINTER(Refine), vp, C.c_int32, vp, vp, vp, C.c_int32]
    L.kpo_refine_cost.restype = C.c_double
    L.kpo_refine_grad.argtypes = [C.POINTER(Problem), C.POINTER(Refine), vp, C.c_int32, vp, vp, vp, C.c_int32, vp]
    L.kpo_refine_grad.restype = C.c_double
    L.kpo_validate_controls.argtypes = [C.POINTER(Problem), vp, vp, vp, C.c_int32, vp, vp, vp, vp]
    L.kpo_validate_controls.restype = C.c_int32


class Refine(C.Structure):
    """Weights of the refinement objective (kpx_oracle.h)."""
    _fields_ = [("w_obs", C.c_double), ("beta", C.c_double), ("margin", C.c_double), ("w_goal", C.c_double),
                ("goal", C.c_double * 3), ("w_effort", C.c_double)]


class OracleProblem:
    """A scene description converted to the oracle's own C struct.

    Holds the FP64 obstacle array alive for as long as the struct is used.
    """

    def __init__(self, prob):
        self.src = prob
        s = Problem()
        s.dyn, s.integ = int(prob.dyn), int(prob.integ)
        s.n, s.m = int(prob.n), int(prob.m)
        s.h = float(prob.h)
        s.k_min, s.k_max = int(prob.k_min), int(prob.k_max)
        for i in range(prob.m):
            s.u_lo[i] = prob.u_lo[i]
            s.u_hi[i] = prob.u_hi[i]
        for i in range(prob.n):
            s.x_lo[i] = prob.x_lo[i]
            s.x_hi[i] = prob.x_hi[i]
        for i, v in enumerate(prob.param):
            s.param[i] = v
        for a in range(3):
            s.ws_lo[a], s.ws_hi[a] = prob.ws_lo[a], prob.ws_hi[a]
            s.goal_c[a] = prob.goal_c[a]
        s.goal_r = prob.goal_r
        s.cost_kind = int(prob.cost_kind)
        s.w_effort = float(prob.w_effort)
        s.n_axes = len(prob.axes)
        for i, ax in enumerate(prob.axes):
            s.ax_dim[i], s.ax_bins[i], s.ax_wrap[i] = ax.state_dim, ax.bins, int(bool(ax.wrap))
            s.ax_lo[i], s.ax_hi[i] = ax.lo, ax.hi
        s.tree_cap, s.lam, s.i_max = int(prob.tree_cap), int(prob.lam), int(prob.i_max)
        self.obs = np.ascontiguousarray(np.asarray(prob.obstacles, dtype=np.float64).reshape(-1, 6))
        s.n_obs = self.obs.shape[0]
        s.seed = int(prob.seed) & 0xFFFFFFFFFFFFFFFF
        s.obs = _p(self.obs, C.c_double)
        self.s = s
        self.n, self.m = s.n, s.m
        self.R = int(np.prod([ax.bins for ax in prob.axes]))

    @property
    def ref(self):
        return C.byref(self.s)


def as_oracle(prob) -> OracleProblem:
    return prob if isinstance(prob, OracleProblem) else OracleProblem(prob)


# ---------------------------------------------------------------------------
# primitive wrappers
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().kpo_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def sample_control(prob, it, node, s):
    P = as_oracle(prob)
    u = np.zeros(8, dtype=np.float32)
    K = np.zeros(1, dtype=np.int32)
    lib().kpo_sample_control(P.ref, it, node, s, u.ctypes.data, K.ctypes.data)
    return u[:P.m].copy(), int(K[0])


def deriv(prob, x, u) -> np.ndarray:
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    dx = np.zeros(P.n)
    lib().kpo_deriv(P.ref, x.ctypes.data, u.ctypes.data, dx.ctypes.data)
    return dx


def step(prob, x, u) -> np.ndarray:
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    xn = np.zeros(P.n)
    lib().kpo_step(P.ref, x.ctypes.data, u.ctypes.data, xn.ctypes.data)
    return xn


def point_valid(prob, x) -> bool:
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return bool(lib().kpo_point_valid(P.ref, x.ctypes.data))


def point_margin(prob, x) -> float:
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().kpo_point_margin(P.ref, x.ctypes.data))


def point_clearance(prob, x) -> float:
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().kpo_point_clearance(P.ref, x.ctypes.data))


def rollout(prob, x0, u, K, traj=False):
    """PropagateODE + validity + edge cost.  Returns a dict."""
    P = as_oracle(prob)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float32).reshape(-1))
    xe = np.zeros(P.n)
    ec = np.zeros(1)
    fb = np.zeros(1, dtype=np.int32)
    mm = np.zeros(1)
    tr = np.zeros((K + 1, P.n)) if traj else None
    v = lib().kpo_rollout(P.ref, x0.ctypes.data, u.ctypes.data, int(K), xe.ctypes.data, ec.ctypes.data,
                          fb.ctypes.data, mm.ctypes.data, tr.ctypes.data if traj else None)
    return dict(valid=bool(v), x_end=xe, edge_cost=float(ec[0]), first_bad=int(fb[0]),
                margin=float(mm[0]), traj=tr)


def region(prob, x):
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    mg = np.zeros(1)
    r = lib().kpo_region(P.ref, x.ctypes.data, mg.ctypes.data)
    return int(r), float(mg[0])


def in_goal(prob, x):
    P = as_oracle(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    mg = np.zeros(1)
    g = lib().kpo_in_goal(P.ref, x.ctypes.data, mg.ctypes.data)
    return bool(g), float(mg[0])


def pack_key(cost: float, node_id: int) -> int:
    return int(lib().kpo_pack_key(float(np.float32(cost)), int(node_id)))


def key_cost(key) -> np.ndarray:
    k = np.asarray(key, dtype=np.uint64)
    return (k >> np.uint64(32)).astype(np.uint32).view(np.float32)


def propagate(prob, it, lam, tree_x, tree_cost, VA, count_A, slots=None):
    """Alg. 2 for the given slots (default: all count_A * lam slots)."""
    P = as_oracle(prob)
    tree_x = np.ascontiguousarray(tree_x, dtype=np.float64)
    tree_cost = np.ascontiguousarray(tree_cost, dtype=np.float64)
    VA = np.ascontiguousarray(VA, dtype=np.int32)
    if slots is None:
        ns = int(count_A) * int(lam)
        sl = None
    else:
        sl = np.ascontiguousarray(slots, dtype=np.int64)
        ns = sl.shape[0]
    out = dict(valid=np.zeros(ns, np.uint8), x_end=np.zeros((ns, P.n)), cost=np.zeros(ns),
               region=np.zeros(ns, np.int32), key=np.zeros(ns, np.uint64), K=np.zeros(ns, np.int32),
               u=np.zeros((ns, P.m), np.float32), vmargin=np.zeros(ns), rmargin=np.zeros(ns),
               in_goal=np.zeros(ns, np.uint8), gmargin=np.zeros(ns))
    o = out
    lib().kpo_propagate(P.ref, int(it), int(lam), tree_x.ctypes.data, tree_cost.ctypes.data,
                        VA.ctypes.data, int(count_A), ns, sl.ctypes.data if sl is not None else None,
                        o["valid"].ctypes.data, o["x_end"].ctypes.data, o["cost"].ctypes.data,
                        o["region"].ctypes.data, o["key"].ctypes.data, o["K"].ctypes.data,
                        o["u"].ctypes.data, o["vmargin"].ctypes.data, o["rmargin"].ctypes.data,
                        o["in_goal"].ctypes.data, o["gmargin"].ctypes.data)
    o["slot"] = np.arange(ns, dtype=np.int64) if sl is None else sl.copy()
    return o


def select_winners(region_key, region_snap, valid, region_, key, n_nodes, tree_cap):
    """Region argmin + V_U filter + capacity.  Returns (region_key, winner idx, n_kept, full)."""
    rk = np.ascontiguousarray(region_key, dtype=np.uint64).copy()
    snap = np.ascontiguousarray(region_snap, dtype=np.uint64)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    region_ = np.ascontiguousarray(region_, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    nc = valid.shape[0]
    win = np.zeros(max(nc, 1), dtype=np.int64)
    nw = np.zeros(1, np.int64)
    nk = np.zeros(1, np.int64)
    full = lib().kpo_select_winners(rk.shape[0], rk.ctypes.data, snap.ctypes.data, nc, valid.ctypes.data,
                                    region_.ctypes.data, key.ctypes.data, int(n_nodes), int(tree_cap),
                                    win.ctypes.data, nw.ctypes.data, nk.ctypes.data)
    return rk, win[:int(nw[0])].copy(), int(nk[0]), bool(full)


def prune(key, region_, parent, set_, icount, region_key, i_max):
    """PruneNodes (Alg. 3).  Returns new (set, icount)."""
    key = np.ascontiguousarray(key, dtype=np.uint64)
    region_ = np.ascontiguousarray(region_, dtype=np.int32)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    s = np.ascontiguousarray(set_, dtype=np.uint8).copy()
    ic = np.ascontiguousarray(icount, dtype=np.uint8).copy()
    rk = np.ascontiguousarray(region_key, dtype=np.uint64)
    lib().kpo_prune(key.shape[0], key.ctypes.data, region_.ctypes.data, parent.ctypes.data, s.ctypes.data,
                    ic.ctypes.data, rk.ctypes.data, int(i_max))
    return s, ic


def append(prob, n_nodes, cand, tree, region_key, goal_key):
    """UpdateTree (Alg. 4) for one iteration's kept winners (kpo_append).
    cand: arrays in slot order -- x [k][n], u [k][m], K, parent, cost (the
    accumulated cost), region, goal (end state in the goal set).  tree: the
    tree arrays x [N][n], u [N][m], K, parent, cost, key, region, set,
    icount.  Returns (tree, region_key, goal_key, first_solution), the inputs
    left unchanged."""
    P = as_oracle(prob)
    k = int(np.asarray(cand["K"]).shape[0])
    cx = np.ascontiguousarray(cand["x"], dtype=np.float64).reshape(k, P.n)
    cu = np.ascontiguousarray(cand["u"], dtype=np.float32).reshape(k, P.m)
    cK = np.ascontiguousarray(cand["K"], dtype=np.int32)
    cp = np.ascontiguousarray(cand["parent"], dtype=np.int32)
    cc = np.ascontiguousarray(cand["cost"], dtype=np.float64)
    cr = np.ascontiguousarray(cand["region"], dtype=np.int32)
    cg = np.ascontiguousarray(cand["goal"], dtype=np.uint8)
    types = dict(x=np.float64, u=np.float32, K=np.int32, parent=np.int32, cost=np.float64, key=np.uint64,
                 region=np.int32, set=np.uint8, icount=np.uint8)
    t = {name: np.ascontiguousarray(tree[name], dtype=dt).copy() for name, dt in types.items()}
    rk = np.ascontiguousarray(region_key, dtype=np.uint64).copy()
    gk = np.array([goal_key], dtype=np.uint64)
    first = lib().kpo_append(P.ref, int(n_nodes), k, cx.ctypes.data, cu.ctypes.data, cK.ctypes.data,
                             cp.ctypes.data, cc.ctypes.data, cr.ctypes.data, cg.ctypes.data, t["x"].ctypes.data,
                             t["u"].ctypes.data, t["K"].ctypes.data, t["parent"].ctypes.data, t["cost"].ctypes.data,
                             t["key"].ctypes.data, t["region"].ctypes.data, t["set"].ctypes.data,
                             t["icount"].ctypes.data, rk.ctypes.data, gk.ctypes.data)
    return t, rk, int(gk[0]), bool(first)


def compact(mask):
    """Exclusive scan + GraphSearch (Alg. 5).  Returns (S, I, count)."""
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
    n = m.shape[0]
    S = np.zeros(n, np.int32)
    I = np.full(n, -1, np.int32)
    cnt = lib().kpo_compact(n, m.ctypes.data, S.ctypes.data, I.ctypes.data)
    return S, I[:cnt].copy(), int(cnt)


def revalidate(prob, states, controls, steps):
    P = as_oracle(prob)
    st = np.ascontiguousarray(states, dtype=np.float64)
    ct = np.ascontiguousarray(controls, dtype=np.float32)
    sp = np.ascontiguousarray(steps, dtype=np.int32)
    L = sp.shape[0]
    out = np.zeros(5)
    ok = lib().kpo_revalidate(P.ref, L, st.ctypes.data, ct.ctypes.data, sp.ctypes.data,
                              out[0:].ctypes.data, out[1:].ctypes.data, out[2:].ctypes.data,
                              out[3:].ctypes.data, out[4:].ctypes.data)
    return dict(ok=bool(ok), max_seg_err=out[0], min_clearance=out[1], goal_slack=out[2],
                cost=out[3], openloop_err=out[4])


class Planner:
    """The oracle's own planner (Alg. 1) on a scene."""

    def __init__(self, prob):
        self.P = as_oracle(prob)
        start = np.ascontiguousarray(np.asarray(prob.start if not isinstance(prob, OracleProblem)
                                                else prob.src.start, dtype=np.float64))
        self.h = lib().kpo_create(self.P.ref, start.ctypes.data)
        if not self.h:
            raise ValueError("oracle planner rejected the problem")

    def __del__(self):
        if getattr(self, "h", None):
            lib().kpo_destroy(self.h)
            self.h = None

    def iterate(self, n=1) -> int:
        return int(lib().kpo_iterate(self.h, int(n)))

    def view(self) -> View:
        v = View()
        lib().kpo_view_state(self.h, C.byref(v))
        return v

    def state(self) -> dict:
        """Copies of the tree arrays (first n_nodes rows) and counters."""
        v = self.view()
        nn, N, R = v.n_nodes, v.N, v.R

        def arr(ptr, count, dt, shape=None):
            a = np.ctypeslib.as_array(ptr, shape=(count,)).astype(dt, copy=True)
            return a.reshape(shape) if shape else a
        return dict(
            n_nodes=nn, count_A=v.count_A, iter=v.iter, tree_full=bool(v.tree_full),
            goal_key=int(v.goal_key), first_solution_iter=v.first_solution_iter, last_lambda=v.last_lambda,
            last_candidates=v.last_candidates, last_valid=v.last_valid, last_winners=v.last_winners,
            total_candidates=v.total_candidates, total_valid=v.total_valid, total_winners=v.total_winners,
            x=arr(v.x, nn * v.n, np.float64, (nn, v.n)) if nn else np.zeros((0, v.n)),
            u=arr(v.u, nn * v.m, np.float32, (nn, v.m)) if nn else np.zeros((0, v.m), np.float32),
            K=arr(v.K, nn, np.int32), parent=arr(v.parent, nn, np.int32), cost=arr(v.cost, nn, np.float64),
            key=arr(v.key, nn, np.uint64), region=arr(v.region, nn, np.int32),
            set=arr(v.set, nn, np.uint8), icount=arr(v.icount, nn, np.uint8),
            region_key=arr(v.region_key, R, np.uint64),
            VA=arr(v.VA, v.count_A, np.int32) if v.count_A else np.zeros(0, np.int32),
        )

    def best_trajectory(self):
        v = self.view()
        cap = v.n_nodes + 1
        st = np.zeros((cap + 1, v.n))
        ct = np.zeros((cap, v.m), np.float32)
        sp = np.zeros(cap, np.int32)
        ln = np.zeros(1, np.int32)
        cost = np.zeros(1)
        rc = lib().kpo_best_trajectory(self.h, cap, st.ctypes.data, ct.ctypes.data, sp.ctypes.data,
                                       ln.ctypes.data, cost.ctypes.data)
        if rc != OK:
            return None
        L = int(ln[0])
        return dict(states=st[:L + 1].copy(), controls=ct[:L].copy(), steps=sp[:L].copy(), cost=float(cost[0]))


def remap_regions(prob, x, key, set_):
    """Region ids, region keys, dominated flags and cell margins of the
    nodes (x[n_nodes][n], key, set) under prob's region grid."""
    P = as_oracle(prob)
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, P.n))
    key = np.ascontiguousarray(key, dtype=np.uint64)
    st = np.ascontiguousarray(set_, dtype=np.uint8)
    nn = x.shape[0]
    region = np.zeros(nn, np.int32)
    rk = np.zeros(P.R, np.uint64)
    dom = np.zeros(nn, np.uint8)
    mg = np.zeros(nn)
    lib().kpo_remap_regions(P.ref, nn, x.ctypes.data, key.ctypes.data, st.ctypes.data, region.ctypes.data,
                            rk.ctypes.data, dom.ctypes.data, mg.ctypes.data)
    return dict(region=region, region_key=rk, dominated=dom.astype(bool), margin=mg)


# ---------------------------------------------------------------------------
# refinement objective (adjoint post-pass reference)
# ---------------------------------------------------------------------------
def _refine_struct(spec) -> Refine:
    r = Refine()
    r.w_obs, r.beta, r.margin, r.w_goal = (float(spec["w_obs"]), float(spec["beta"]), float(spec["margin"]),
                                           float(spec["w_goal"]))
    for a in range(3):
        r.goal[a] = float(spec["goal"][a])
    r.w_effort = float(spec["w_effort"])
    return r


def box_distance(box, p):
    """Signed distance from p to a closed box (negative inside) and its gradient."""
    b = np.ascontiguousarray(box, dtype=np.float64)
    q = np.ascontiguousarray(p, dtype=np.float64)
    g = np.zeros(3)
    d = lib().kpo_box_distance(b.ctypes.data, q.ctypes.data, g.ctypes.data)
    return float(d), g


def _refine_args(prob, x0, u, K, obstacles):
    P = as_oracle(prob)
    obs = P.obs if obstacles is None else np.ascontiguousarray(np.asarray(obstacles, np.float64).reshape(-1, 6))
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4))
    K = np.ascontiguousarray(K, dtype=np.int32)
    return P, obs, x0, u, K


def refine_cost(prob, spec, x0, u, K, obstacles=None) -> float:
    """The refinement objective J of a control sequence u[S][4] held K[s] steps."""
    P, obs, x0, u, K = _refine_args(prob, x0, u, K, obstacles)
    r = _refine_struct(spec)
    return float(lib().kpo_refine_cost(P.ref, C.byref(r), obs.ctypes.data, obs.shape[0], x0.ctypes.data,
                                       u.ctypes.data, K.ctypes.data, K.shape[0]))


def refine_grad(prob, spec, x0, u, K, obstacles=None):
    """(J, dJ/du[S][4]) by plain reverse mode in FP64."""
    P, obs, x0, u, K = _refine_args(prob, x0, u, K, obstacles)
    r = _refine_struct(spec)
    g = np.zeros_like(u)
    J = lib().kpo_refine_grad(P.ref, C.byref(r), obs.ctypes.data, obs.shape[0], x0.ctypes.data, u.ctypes.data,
                              K.ctypes.data, K.shape[0], g.ctypes.data)
    return float(J), g


def validate_controls(prob, x0, u, K):
    """Open-loop FP64 re-validation of FP32 controls u[S][m] from x0."""
    P = as_oracle(prob)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    uf = np.ascontiguousarray(np.asarray(u, dtype=np.float32).reshape(-1))
    K = np.ascontiguousarray(K, dtype=np.int32)
    mc, gd, c = np.zeros(1), np.zeros(1), np.zeros(1)
    xe = np.zeros(P.n)
    ok = lib().kpo_validate_controls(P.ref, x0.ctypes.data, uf.ctypes.data, K.ctypes.data, K.shape[0],
                                     mc.ctypes.data, gd.ctypes.data, c.ctypes.data, xe.ctypes.data)
    return dict(valid=bool(ok), min_clearance=float(mc[0]), goal_dist=float(gd[0]), cost=float(c[0]), x_end=xe)

