"""Python binding of libkpx.so, the GB300 Kino-PAX+ planning library.

Thin argument marshalling over the C ABI of include/kpx.h (ctypes): the
functions below carry the C names and every step of the planning iteration
runs in the library's CUDA kernels.  PyTorch provides the device workspace
(a uint8 tensor owned by the ``Planner``) and the CUDA stream.

The library is loaded on first use; if it has not been built, or cannot be
loaded, a RuntimeError is raised.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading
from typing import Optional

import numpy as np

from . import scenes  # noqa: F401  (re-exported for convenience)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkpx.so")
_lock = threading.Lock()
_lib = None

# status codes (kpx_status)
KPX_OK, KPX_E_INVALID, KPX_E_NOMEM, KPX_E_CUDA = 0, 1, 2, 3
KPX_TREE_FULL, KPX_NO_SOLUTION, KPX_E_TIMEOUT, KPX_E_INTERNAL = 4, 5, 6, 7
KPX_FLAG_EARLY_REJECT = 1
KPX_FLAG_NO_FUSED = 2
KPX_FLAG_NO_SLOT_ORDER = 4
PHASES = ("begin", "propagate", "mark", "scan", "append", "prune", "end")
KEY_INF = 0xFFFFFFFFFFFFFFFF

EXPORTED = ("kpx_workspace_size", "kpx_create", "kpx_iterate", "kpx_best_trajectory", "kpx_reset",
            "kpx_destroy", "kpx_status_str", "kpx_last_error", "kpx_get_layout", "kpx_debug_step",
            "kpx_snapshot", "kpx_restore", "kpx_plan_static", "kpx_batch_workspace_size", "kpx_batch_create",
            "kpx_batch_iterate", "kpx_batch_member", "kpx_batch_reset", "kpx_batch_destroy", "kpx_batch_last_error",
            "kpx_batch_assign", "kpx_batch_release", "kpx_batch_poll", "kpx_graph_info",
            "kpx_refine_workspace_size", "kpx_refine_eval", "kpx_refine_validate", "kpx_refine_adam",
            "kpx_refine_keep_best", "kpx_set_launch", "kpx_batch_set_launch", "kpx_set_regions",
            "kpx_fp32_fma_rate", "kpx_refine_counters", "kpx_debug_wait_timeout")


class kpx_dynamics(C.Structure):
    _fields_ = [("kind", C.c_int32), ("integ", C.c_int32), ("h", C.c_float), ("k_min", C.c_int32),
                ("k_max", C.c_int32), ("u_lo", C.c_float * 8), ("u_hi", C.c_float * 8),
                ("x_lo", C.c_float * 16), ("x_hi", C.c_float * 16), ("param", C.c_float * 8)]


class kpx_workspace(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3)]


class kpx_obstacles(C.Structure):
    _fields_ = [("aabb", C.POINTER(C.c_float)), ("count", C.c_int32)]


class kpx_goal(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("radius", C.c_float)]


class kpx_cost(C.Structure):
    _fields_ = [("kind", C.c_int32), ("w_effort", C.c_float)]


class kpx_region_axis(C.Structure):
    _fields_ = [("state_dim", C.c_int32), ("bins", C.c_int32), ("lo", C.c_float), ("hi", C.c_float),
                ("wrap", C.c_int32)]


class kpx_config(C.Structure):
    _fields_ = [("tree_cap", C.c_int32), ("samples_per_node", C.c_int32), ("n_axes", C.c_int32),
                ("axis", kpx_region_axis * 8), ("i_max", C.c_int32), ("seed", C.c_uint64),
                ("flags", C.c_int32), ("region_capacity", C.c_int32)]


class kpx_iter_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iter", C.c_int32), ("n_nodes", C.c_int32), ("n_active", C.c_int32),
                ("n_inactive", C.c_int32), ("n_terminal", C.c_int32), ("lam", C.c_int32),
                ("first_solution_iter", C.c_int32), ("candidates", C.c_int64), ("valid", C.c_int64),
                ("winners", C.c_int64), ("total_candidates", C.c_int64), ("total_valid", C.c_int64),
                ("total_winners", C.c_int64), ("best_cost", C.c_float), ("pad", C.c_float),
                ("first_solution_ns", C.c_uint64), ("elapsed_ns", C.c_uint64),
                ("total_steps", C.c_uint64), ("total_box_tests", C.c_uint64)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "pad"}


class kpx_device_header(C.Structure):
    _fields_ = [("status", C.c_int32), ("active", C.c_int32), ("iter", C.c_int32), ("n_nodes", C.c_int32),
                ("count_A", C.c_int32), ("lam", C.c_int32), ("va_sel", C.c_int32),
                ("first_solution_iter", C.c_int32), ("n_slots", C.c_int64), ("goal_key", C.c_uint64),
                ("n_win", C.c_int32), ("n_kept", C.c_int32), ("count_A_next", C.c_int32), ("epoch", C.c_int32),
                ("prop_ticket", C.c_uint64), ("win_ticket", C.c_uint32), ("prune_ticket", C.c_uint32),
                ("n_active", C.c_int32), ("n_inactive", C.c_int32), ("n_terminal", C.c_int32), ("graph_pending", C.c_int32),
                ("last_candidates", C.c_uint64), ("last_valid", C.c_uint64), ("last_winners", C.c_uint64),
                ("total_candidates", C.c_uint64), ("total_valid", C.c_uint64), ("total_winners", C.c_uint64),
                ("t_start_ns", C.c_uint64), ("t_first_solution_ns", C.c_uint64), ("t_last_ns", C.c_uint64),
                ("traj_len", C.c_int32), ("graph_ctl", C.c_int32), ("total_steps", C.c_uint64),
                ("total_box_tests", C.c_uint64), ("err_info", C.c_uint32 * 4), ("fused_iterations", C.c_uint64)]


class kpx_layout(C.Structure):
    _fields_ = [("header", C.c_void_p), ("x", C.c_void_p), ("u", C.c_void_p), ("K", C.c_void_p),
                ("parent", C.c_void_p), ("key", C.c_void_p), ("region", C.c_void_p), ("set", C.c_void_p),
                ("icount", C.c_void_p), ("region_key", C.c_void_p), ("region_snap", C.c_void_p),
                ("va", C.c_void_p * 2), ("win_slot", C.c_void_p), ("win_mask", C.c_void_p),
                ("obstacles", C.c_void_p), ("n", C.c_int32), ("m", C.c_int32), ("N", C.c_int32),
                ("R", C.c_int32), ("va_cap", C.c_int32), ("n_obstacles", C.c_int32), ("slot_cap", C.c_int64),
                ("mask_words", C.c_int64), ("workspace_bytes", C.c_size_t), ("slot_order", C.c_void_p)]


class kpx_problem(C.Structure):
    _fields_ = [("dyn", C.POINTER(kpx_dynamics)), ("ws", C.POINTER(kpx_workspace)),
                ("obs", C.POINTER(kpx_obstacles)), ("start", C.POINTER(C.c_float)), ("goal", C.POINTER(kpx_goal)),
                ("cost", C.POINTER(kpx_cost)), ("cfg", C.POINTER(kpx_config))]


class kpx_launch_config(C.Structure):
    _fields_ = [("propagate_blocks_per_sm", C.c_int32), ("grid_scale", C.c_float)]


class kpx_slot_state(C.Structure):
    _fields_ = [("status", C.c_int32), ("iter", C.c_int32), ("n_nodes", C.c_int32),
                ("first_solution_iter", C.c_int32), ("goal_key", C.c_uint64), ("t_start_ns", C.c_uint64),
                ("t_first_solution_ns", C.c_uint64), ("t_last_ns", C.c_uint64), ("t_poll_ns", C.c_uint64)]


class kpx_debug_records(C.Structure):
    _fields_ = [("valid", C.c_void_p), ("region", C.c_void_p), ("key", C.c_void_p), ("K", C.c_void_p),
                ("x", C.c_void_p), ("u", C.c_void_p), ("capacity", C.c_int64)]


def load(path: Optional[str] = None):
    """Load libkpx.so (built by __graft_entry__.build() or ``python -m
    paper_2602_02846_gb300.build``).  Raises RuntimeError if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("libkpx.so is not built (%s); run __graft_entry__.build() first" % p)
        try:
            L = C.CDLL(p)
        except OSError as e:
            raise RuntimeError("cannot load libkpx.so: %s" % e) from e
        vp = C.c_void_p
        L.kpx_workspace_size.argtypes = [C.POINTER(kpx_dynamics), C.POINTER(kpx_config), C.c_int32]
        L.kpx_workspace_size.restype = C.c_size_t
        L.kpx_create.argtypes = [C.POINTER(kpx_dynamics), C.POINTER(kpx_workspace), C.POINTER(kpx_obstacles),
                                 C.POINTER(C.c_float), C.POINTER(kpx_goal), C.POINTER(kpx_cost),
                                 C.POINTER(kpx_config), vp, C.c_size_t, vp, C.POINTER(vp)]
        L.kpx_create.restype = C.c_int
        L.kpx_iterate.argtypes = [vp, C.c_int32, C.POINTER(kpx_iter_stats)]
        L.kpx_iterate.restype = C.c_int
        L.kpx_best_trajectory.argtypes = [vp, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_float)]
        L.kpx_best_trajectory.restype = C.c_int
        L.kpx_reset.argtypes = [vp]
        L.kpx_reset.restype = C.c_int
        L.kpx_destroy.argtypes = [vp]
        L.kpx_destroy.restype = C.c_int
        L.kpx_status_str.argtypes = [C.c_int]
        L.kpx_status_str.restype = C.c_char_p
        L.kpx_last_error.argtypes = [vp]
        L.kpx_last_error.restype = C.c_char_p
        L.kpx_get_layout.argtypes = [vp, C.POINTER(kpx_layout)]
        L.kpx_get_layout.restype = C.c_int
        L.kpx_debug_step.argtypes = [vp, C.c_int32, C.POINTER(kpx_debug_records)]
        L.kpx_debug_step.restype = C.c_int
        L.kpx_snapshot.argtypes = [vp, vp]
        L.kpx_snapshot.restype = C.c_int
        L.kpx_restore.argtypes = [vp, vp]
        L.kpx_restore.restype = C.c_int
        L.kpx_plan_static.argtypes = [C.POINTER(kpx_dynamics), C.POINTER(kpx_workspace), C.POINTER(kpx_obstacles),
                                      C.POINTER(C.c_float), C.POINTER(kpx_goal), C.POINTER(kpx_cost),
                                      C.POINTER(kpx_config), C.c_int32, vp, C.c_int32, C.POINTER(C.c_float),
                                      C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_float)]
        L.kpx_plan_static.restype = C.c_int
        L.kpx_batch_workspace_size.argtypes = [C.c_int32, C.POINTER(kpx_problem)]
        L.kpx_batch_workspace_size.restype = C.c_size_t
        L.kpx_batch_create.argtypes = [C.c_int32, C.POINTER(kpx_problem), vp, C.c_size_t, vp, C.POINTER(vp)]
        L.kpx_batch_create.restype = C.c_int
        L.kpx_batch_iterate.argtypes = [vp, C.c_int32]
        L.kpx_batch_iterate.restype = C.c_int
        L.kpx_batch_member.argtypes = [vp, C.c_int32, C.POINTER(vp)]
        L.kpx_batch_member.restype = C.c_int
        L.kpx_batch_reset.argtypes = [vp]
        L.kpx_batch_reset.restype = C.c_int
        L.kpx_batch_destroy.argtypes = [vp]
        L.kpx_batch_destroy.restype = C.c_int
        L.kpx_batch_last_error.argtypes = [vp]
        L.kpx_batch_last_error.restype = C.c_char_p
        L.kpx_batch_assign.argtypes = [vp, C.c_int32, C.POINTER(kpx_problem), C.c_int32, vp, C.c_size_t]
        L.kpx_batch_assign.restype = C.c_int
        L.kpx_batch_release.argtypes = [vp, C.c_int32]
        L.kpx_batch_release.restype = C.c_int
        L.kpx_batch_poll.argtypes = [vp, C.POINTER(kpx_slot_state)]
        L.kpx_batch_poll.restype = C.c_int
        L.kpx_graph_info.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.kpx_graph_info.restype = C.c_int
        L.kpx_debug_wait_timeout.argtypes = [vp]
        L.kpx_debug_wait_timeout.restype = C.c_int
        L.kpx_refine_counters.argtypes = [vp, C.POINTER(C.c_uint64), vp]
        L.kpx_refine_counters.restype = C.c_int
        L.kpx_fp32_fma_rate.argtypes = [C.c_int32, C.POINTER(C.c_double), vp]
        L.kpx_fp32_fma_rate.restype = C.c_int
        L.kpx_set_regions.argtypes = [vp, C.c_int32, C.POINTER(kpx_region_axis)]
        L.kpx_set_regions.restype = C.c_int
        L.kpx_set_launch.argtypes = [vp, C.POINTER(kpx_launch_config)]
        L.kpx_set_launch.restype = C.c_int
        L.kpx_batch_set_launch.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(kpx_launch_config)]
        L.kpx_batch_set_launch.restype = C.c_int
        _lib = L
        return L


class KpxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("kpx status %d (%s): %s" % (status, _status_name(status), msg))
        self.status = status


def _status_name(s):
    try:
        return load().kpx_status_str(int(s)).decode()
    except Exception:
        return "?"


# ---------------------------------------------------------------------------
# marshalling of a scene description (scenes.Problem) into the C structs
# ---------------------------------------------------------------------------
def problem_structs(prob, flags: int = 0):
    d = kpx_dynamics()
    d.kind, d.integ, d.h = int(prob.dyn), int(prob.integ), float(prob.h)
    d.k_min, d.k_max = int(prob.k_min), int(prob.k_max)
    for i in range(prob.m):
        d.u_lo[i], d.u_hi[i] = prob.u_lo[i], prob.u_hi[i]
    for i in range(prob.n):
        d.x_lo[i], d.x_hi[i] = prob.x_lo[i], prob.x_hi[i]
    for i, v in enumerate(prob.param):
        d.param[i] = v
    w = kpx_workspace()
    for a in range(3):
        w.lo[a], w.hi[a] = prob.ws_lo[a], prob.ws_hi[a]
    g = kpx_goal()
    for a in range(3):
        g.center[a] = prob.goal_c[a]
    g.radius = prob.goal_r
    c = kpx_cost()
    c.kind, c.w_effort = int(prob.cost_kind), float(prob.w_effort)
    cfg = kpx_config()
    cfg.tree_cap, cfg.samples_per_node, cfg.n_axes = int(prob.tree_cap), int(prob.lam), len(prob.axes)
    for i, ax in enumerate(prob.axes):
        cfg.axis[i].state_dim, cfg.axis[i].bins = ax.state_dim, ax.bins
        cfg.axis[i].lo, cfg.axis[i].hi, cfg.axis[i].wrap = ax.lo, ax.hi, int(bool(ax.wrap))
    cfg.i_max = int(prob.i_max)
    cfg.seed = int(prob.seed) & 0xFFFFFFFFFFFFFFFF
    cfg.flags = int(flags)
    cfg.region_capacity = int(prob.region_capacity)
    obs = np.ascontiguousarray(np.asarray(prob.obstacles, dtype=np.float32).reshape(-1, 6))
    o = kpx_obstacles()
    o.aabb = obs.ctypes.data_as(C.POINTER(C.c_float))
    o.count = obs.shape[0]
    start = np.ascontiguousarray(np.asarray(prob.start, dtype=np.float32))
    return d, w, o, g, c, cfg, obs, start


def kpx_workspace_size(prob, flags: int = 0) -> int:
    """Device bytes kpx_create needs for ``prob`` (0 if the problem is invalid)."""
    d, w, o, g, c, cfg, obs, start = problem_structs(prob, flags)
    return int(load().kpx_workspace_size(C.byref(d), C.byref(cfg), o.count))


class Planner:
    """One planning problem on one GPU (kpx_create ... kpx_destroy).

    The device workspace is a torch uint8 tensor owned by this object; work
    runs on ``stream`` (default: the current torch stream of ``device``).
    """

    def __init__(self, prob, device=None, stream=None, flags: int = 0, workspace=None):
        import torch
        L = load()
        self.prob = prob
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        d, w, o, g, c, cfg, obs, start = problem_structs(prob, flags)
        self._structs = (d, w, o, g, c, cfg, obs, start)
        size = int(L.kpx_workspace_size(C.byref(d), C.byref(cfg), o.count))
        if size == 0:
            raise KpxError(KPX_E_INVALID, "problem rejected by kpx_workspace_size")
        if workspace is not None:
            if workspace.dtype != torch.uint8 or workspace.numel() < size + 256 or not workspace.is_cuda:
                raise KpxError(KPX_E_NOMEM, "workspace tensor must be CUDA uint8 of >= %d bytes" % (size + 256))
            self.workspace = workspace
        else:
            self.workspace = torch.empty(size + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._off = (-base) % 256
        self.ws_ptr = base + self._off
        self.ws_bytes = size
        h = C.c_void_p()
        st = L.kpx_create(C.byref(d), C.byref(w), C.byref(o), start.ctypes.data_as(C.POINTER(C.c_float)),
                          C.byref(g), C.byref(c), C.byref(cfg), C.c_void_p(self.ws_ptr), C.c_size_t(size),
                          C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != KPX_OK:
            raise KpxError(st, L.kpx_last_error(None).decode())
        self.h = h
        self.n, self.m = prob.n, prob.m

    # -- C ABI calls ----------------------------------------------------------
    def _check(self, st, ok=(KPX_OK,)):
        if st not in ok:
            raise KpxError(st, load().kpx_last_error(self.h).decode())
        return st

    def iterate(self, n_iters: int = 1, stats: bool = False):
        """kpx_iterate: asynchronous unless stats are requested."""
        L = load()
        if stats:
            s = kpx_iter_stats()
            st = L.kpx_iterate(self.h, int(n_iters), C.byref(s))
            self._check(st, (KPX_OK, KPX_TREE_FULL))
            return s.as_dict()
        self._check(L.kpx_iterate(self.h, int(n_iters), None))
        return None

    def best_trajectory(self, capacity: Optional[int] = None):
        """kpx_best_trajectory: dict(states, controls, steps, cost) or None."""
        L = load()
        cap = int(capacity if capacity is not None else 1024)
        while True:
            states = np.zeros((cap + 1, self.n), np.float32)
            controls = np.zeros((cap, self.m), np.float32)
            steps = np.zeros(cap, np.int32)
            ln = C.c_int32(0)
            cost = C.c_float(0)
            st = L.kpx_best_trajectory(self.h, cap, states.ctypes.data_as(C.POINTER(C.c_float)),
                                       controls.ctypes.data_as(C.POINTER(C.c_float)),
                                       steps.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(ln), C.byref(cost))
            if st == KPX_NO_SOLUTION:
                return None
            if st == KPX_E_INVALID and ln.value > cap and capacity is None:
                cap = ln.value
                continue
            self._check(st)
            k = ln.value
            return dict(states=states[:k + 1], controls=controls[:k], steps=steps[:k], cost=float(cost.value))

    def reset(self):
        self._check(load().kpx_reset(self.h))

    def set_regions(self, axes):
        """kpx_set_regions: a new region decomposition (scenes.RegionAxis list)."""
        arr = (kpx_region_axis * max(1, len(axes)))()
        for i, ax in enumerate(axes):
            arr[i].state_dim, arr[i].bins = int(ax.state_dim), int(ax.bins)
            arr[i].lo, arr[i].hi, arr[i].wrap = float(ax.lo), float(ax.hi), int(bool(ax.wrap))
        self._check(load().kpx_set_regions(self.h, len(axes), arr))
        self.prob = dataclasses.replace(self.prob, axes=list(axes)) if dataclasses.is_dataclass(self.prob) else self.prob

    def set_launch(self, blocks_per_sm: int = 0, grid_scale: float = 0.0):
        """kpx_set_launch: launch choices that leave results unchanged."""
        lc = kpx_launch_config(int(blocks_per_sm), float(grid_scale))
        self._check(load().kpx_set_launch(self.h, C.byref(lc)))

    def graph_info(self):
        """kpx_graph_info: (max iterations per graph launch, fused)."""
        mx, fu = C.c_int32(), C.c_int32()
        self._check(load().kpx_graph_info(self.h, C.byref(mx), C.byref(fu)))
        return int(mx.value), bool(fu.value)

    @staticmethod
    def launch_plan(n_iters: int, max_per_launch: int):
        """Iterations per graph launch of kpx_iterate(n_iters) (kpx_graph_info:
        one launch per call, up to max_per_launch iterations each)."""
        out, left = [], int(n_iters)
        while left > 0 and max_per_launch > 0:
            g = min(left, max_per_launch)
            out.append(g)
            left -= g
        return out

    def close(self):
        if getattr(self, "_borrowed", False):
            self.h = None
            return
        if getattr(self, "h", None):
            load().kpx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self) -> kpx_layout:
        lay = kpx_layout()
        self._check(load().kpx_get_layout(self.h, C.byref(lay)))
        return lay

    def debug_step(self, phase, records: Optional[dict] = None):
        """kpx_debug_step for one phase (name or index); records: dict of
        torch tensors from ``make_records``."""
        ph = PHASES.index(phase) if isinstance(phase, str) else int(phase)
        rp = None
        if records is not None:
            r = kpx_debug_records()
            r.valid, r.region, r.key = records["valid"].data_ptr(), records["region"].data_ptr(), records["key"].data_ptr()
            r.K, r.x, r.u = records["K"].data_ptr(), records["x"].data_ptr(), records["u"].data_ptr()
            r.capacity = records["capacity"]
            rp = C.byref(r)
        self._check(load().kpx_debug_step(self.h, ph, rp))

    def make_records(self):
        import torch
        cap = int(self.layout().slot_cap)
        dev = self.device
        return dict(valid=torch.zeros(cap, dtype=torch.uint8, device=dev),
                    region=torch.zeros(cap, dtype=torch.int32, device=dev),
                    key=torch.zeros(cap, dtype=torch.int64, device=dev),
                    K=torch.zeros(cap, dtype=torch.int32, device=dev),
                    x=torch.zeros(self.n * cap, dtype=torch.float32, device=dev),
                    u=torch.zeros(self.m * cap, dtype=torch.float32, device=dev),
                    capacity=cap)

    def snapshot(self):
        """kpx_snapshot into a device tensor (a full copy of the workspace)."""
        import torch
        buf = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self._check(load().kpx_snapshot(self.h, C.c_void_p(buf.data_ptr())))
        return buf

    def restore(self, buf):
        self._check(load().kpx_restore(self.h, C.c_void_p(buf.data_ptr())))

    # -- read-only views of the device arrays (for tests and inspection) -----
    def _view(self, ptr, nbytes, dtype):
        off = int(ptr) - self.ws_ptr + self._off
        return self.workspace[off:off + nbytes].view(dtype)

    def header(self) -> kpx_device_header:
        lay = self.layout()
        self.stream.synchronize()
        raw = self._view(lay.header, C.sizeof(kpx_device_header), __import__("torch").uint8).cpu().numpy()
        return kpx_device_header.from_buffer_copy(raw.tobytes())

    def arrays(self, n_nodes: Optional[int] = None) -> dict:
        """Host copies of the tree arrays (first n_nodes rows) and region keys."""
        import torch
        lay = self.layout()
        h = self.header()
        nn = h.n_nodes if n_nodes is None else n_nodes
        N, R = lay.N, lay.R
        x = self._view(lay.x, 4 * self.n * N, torch.float32).view(self.n, N)[:, :nn].T.cpu().numpy()
        u = self._view(lay.u, 4 * self.m * N, torch.float32).view(self.m, N)[:, :nn].T.cpu().numpy()
        K = self._view(lay.K, 2 * N, torch.int16)[:nn].cpu().numpy().astype(np.int32) & 0xFFFF
        parent = self._view(lay.parent, 4 * N, torch.int32)[:nn].cpu().numpy()
        key = self._view(lay.key, 8 * N, torch.int64)[:nn].cpu().numpy().view(np.uint64)
        region = self._view(lay.region, 4 * N, torch.int32)[:nn].cpu().numpy()
        setb = self._view(lay.set, N, torch.uint8)[:nn].cpu().numpy()
        icount = self._view(lay.icount, N, torch.uint8)[:nn].cpu().numpy()
        rk = self._view(lay.region_key, 8 * R, torch.int64).cpu().numpy().view(np.uint64)
        snap = self._view(lay.region_snap, 8 * R, torch.int64).cpu().numpy().view(np.uint64)
        va_ptr = lay.va[h.va_sel]
        va = self._view(va_ptr, 4 * lay.va_cap, torch.int32)[:h.count_A].cpu().numpy()
        return dict(header=h, x=x, u=u, K=K, parent=parent, key=key, region=region, set=setb & 3,
                    set_raw=setb, icount=icount, region_key=rk, region_snap=snap, VA=va,
                    n_nodes=h.n_nodes, count_A=h.count_A, iter=h.iter, goal_key=int(h.goal_key))

    def slot_order(self, n_slots: int) -> np.ndarray:
        """The propagate order of the current iteration (begin phase), as
        offsets within each 128-slot chunk; None when disabled."""
        import torch
        lay = self.layout()
        if not lay.slot_order:
            return None
        self.stream.synchronize()
        total = (int(n_slots) + 127) // 128 * 128
        return self._view(lay.slot_order, total, torch.uint8).cpu().numpy()

    def win_slots(self, count: int) -> np.ndarray:
        import torch
        lay = self.layout()
        return self._view(lay.win_slot, 4 * lay.R, torch.int32)[:count].cpu().numpy()


def _fill_problem(dst, structs):
    d, w, o, g, c, cfg, obs, start = structs
    dst.dyn, dst.ws, dst.obs = C.pointer(d), C.pointer(w), C.pointer(o)
    dst.start = start.ctypes.data_as(C.POINTER(C.c_float))
    dst.goal, dst.cost, dst.cfg = C.pointer(g), C.pointer(c), C.pointer(cfg)


class BatchPlanner:
    """Many independent problems iterated together (kpx_batch_*): every phase
    is one launch for the whole batch.  ``member(i)`` gives a Planner view of
    problem i (statistics, trajectory, arrays) owned by the batch."""

    def __init__(self, problems, device=None, stream=None, flags: int = 0):
        import torch
        L = load()
        self.problems = list(problems)
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.flags = flags
        self._structs = [problem_structs(p, flags) for p in self.problems]
        arr = (kpx_problem * len(self.problems))()
        for i, st in enumerate(self._structs):
            _fill_problem(arr[i], st)
        self._arr = arr
        self._poll = (kpx_slot_state * len(self.problems))()
        size = int(L.kpx_batch_workspace_size(len(self.problems), arr))
        if size == 0:
            raise KpxError(KPX_E_INVALID, "batch rejected by kpx_batch_workspace_size")
        self.workspace = torch.empty(size + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._off = (-base) % 256
        self.ws_ptr = base + self._off
        h = C.c_void_p()
        st = L.kpx_batch_create(len(self.problems), arr, C.c_void_p(self.ws_ptr), C.c_size_t(size),
                                C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != KPX_OK:
            raise KpxError(st, L.kpx_batch_last_error(None).decode())
        self.h = h
        self._members = {}
        self._slot_ws = {}  # slot -> tensor holding its workspace when not the batch's own

    def iterate(self, n_iters: int = 1):
        st = load().kpx_batch_iterate(self.h, int(n_iters))
        if st != KPX_OK:
            raise KpxError(st, load().kpx_batch_last_error(self.h).decode())

    def reset(self):
        st = load().kpx_batch_reset(self.h)
        if st != KPX_OK:
            raise KpxError(st, load().kpx_batch_last_error(self.h).decode())

    def assign(self, i: int, prob, iter_limit: int = 0, workspace=None, offset: int = 0,
               nbytes: Optional[int] = None):
        """Re-initialise slot i with ``prob`` (same dynamics class); it
        iterates with the batch until it has done ``iter_limit`` iterations
        (0: no limit).  ``workspace``: a uint8 device tensor holding the
        slot's tree from byte ``offset`` (256-byte aligned address, ``nbytes``
        bytes, default the rest of the tensor), kept alive by the caller until
        the slot is released; None keeps the slot's current workspace.
        Asynchronous."""
        structs = problem_structs(prob, self.flags)
        one = kpx_problem()
        _fill_problem(one, structs)
        ptr, size = None, 0
        if workspace is not None:
            ptr = workspace.data_ptr() + int(offset)
            size = int(nbytes) if nbytes is not None else workspace.numel() - int(offset)
        st = load().kpx_batch_assign(self.h, int(i), C.byref(one), int(iter_limit), C.c_void_p(ptr),
                                     C.c_size_t(size))
        if st != KPX_OK:
            raise KpxError(st, load().kpx_batch_last_error(self.h).decode())
        self.problems[i] = prob
        self._structs[i] = structs
        if workspace is not None:
            self._slot_ws[i] = workspace
        self._members.pop(i, None)  # the slot's layout follows the new problem

    def release(self, i: int):
        """Mark slot i vacant: work enqueued after this never touches the
        slot's workspace (its arrays stay readable until that memory is
        reused)."""
        st = load().kpx_batch_release(self.h, int(i))
        if st != KPX_OK:
            raise KpxError(st, load().kpx_batch_last_error(self.h).decode())

    def poll(self):
        """Waits for the batch's stream; returns one dict per slot (status -1:
        vacant; goal_cost None: no solution yet)."""
        st = load().kpx_batch_poll(self.h, self._poll)
        if st != KPX_OK:
            raise KpxError(st, load().kpx_batch_last_error(self.h).decode())
        out = []
        for s in self._poll:
            key = int(s.goal_key)
            cost = None if key == KEY_INF else \
                float(np.frombuffer(np.uint32(key >> 32).tobytes(), np.float32)[0])
            out.append({"status": int(s.status), "iter": int(s.iter), "n_nodes": int(s.n_nodes),
                        "first_solution_iter": int(s.first_solution_iter), "goal_cost": cost,
                        "t_start_ns": int(s.t_start_ns), "t_first_solution_ns": int(s.t_first_solution_ns),
                        "t_last_ns": int(s.t_last_ns), "t_poll_ns": int(s.t_poll_ns)})
        return out

    def set_launch(self, dyn: int, integ: int, blocks_per_sm: int = 0, grid_scale: float = 0.0):
        """kpx_batch_set_launch for every problem of dynamics class (dyn, integ)."""
        lc = kpx_launch_config(int(blocks_per_sm), float(grid_scale))
        st = load().kpx_batch_set_launch(self.h, int(dyn), int(integ), C.byref(lc))
        if st != KPX_OK:
            raise KpxError(st, load().kpx_batch_last_error(self.h).decode())

    def autotune(self, iters: int = 4, blocks=(0, 1, 2, 3), scales=(0.5, 0.75, 1.0, 2.0)):
        """Per dynamics class, times ``iters`` batched iterations from the
        current state for every (blocks per SM, grid scale) pair, one class at
        a time with the others at their chosen settings, and keeps the
        fastest.  The batch's state is restored after each trial, so
        planning continues from where it was.  Every choice gives the same
        results.  Needs the batch's problems in its own workspace (not in
        slots reassigned elsewhere).  Returns {(dyn, integ): dict(blocks,
        scale, ms, trials)}."""
        import torch
        classes = sorted({(int(p.dyn), int(p.integ)) for p in self.problems})
        base = {c: (0, 1.0) for c in classes}
        chosen = dict(base)
        snap = self.workspace.clone()
        s = self.stream

        def apply_settings(settings):
            # the restored workspace holds the snapshot's grids: bring the host
            # side back to that scale, then to the trial's (the blocks per SM
            # are host-only and are set once, so the captured graphs stay)
            for c in classes:
                self.set_launch(c[0], c[1], settings[c][0], base[c][1])
                self.set_launch(c[0], c[1], settings[c][0], settings[c][1])

        def run(settings):
            with torch.cuda.stream(s):
                self.workspace.copy_(snap)
            apply_settings(settings)
            self.iterate(iters)  # builds the graphs for these launch shapes
            with torch.cuda.stream(s):
                self.workspace.copy_(snap)
            apply_settings(settings)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            self.iterate(iters)
            b.record(s)
            b.synchronize()
            return a.elapsed_time(b)

        report = {}
        for c in classes:
            trials = []
            for bps in blocks:
                for sc in scales:
                    trial = dict(chosen)
                    trial[c] = (bps, sc)
                    trials.append((run(trial), bps, sc))
            ms, bps, sc = min(trials)
            chosen[c] = (bps, sc)
            report[c] = dict(blocks=bps, scale=sc, ms=ms, trials=[(b_, s_, t_) for t_, b_, s_ in trials])
        with torch.cuda.stream(s):
            self.workspace.copy_(snap)
        apply_settings(chosen)
        s.synchronize()
        return report

    def member(self, i: int) -> "Planner":
        if i in self._members:
            return self._members[i]
        L = load()
        mh = C.c_void_p()
        if L.kpx_batch_member(self.h, int(i), C.byref(mh)) != KPX_OK:
            raise KpxError(KPX_E_INVALID, "no member %d" % i)
        view = Planner.__new__(Planner)
        view.prob = self.problems[i]
        view.device, view.stream = self.device, self.stream
        view.workspace = self._slot_ws.get(i, self.workspace)
        view.h = mh
        view._borrowed = True
        view.n, view.m = self.problems[i].n, self.problems[i].m
        lay = view.layout()
        view.ws_ptr = int(lay.header)
        view._off = view.ws_ptr - view.workspace.data_ptr()
        view.ws_bytes = int(lay.workspace_bytes)
        self._members[i] = view
        return view

    def close(self):
        if getattr(self, "h", None):
            load().kpx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kpx_plan_static(prob, n_iters: int, stream=None, capacity: int = 4096, flags: int = 0):
    """One planning run in the library's static device memory (no
    allocation anywhere; see include/kpx.h).  ``stream``: a torch CUDA stream
    or None for the legacy default stream.  Returns (status, trajectory dict
    or None)."""
    L = load()
    d, w, o, g, c, cfg, obs, start = problem_structs(prob, flags)
    states = np.zeros((capacity + 1, prob.n), np.float32)
    controls = np.zeros((capacity, prob.m), np.float32)
    steps = np.zeros(capacity, np.int32)
    ln = C.c_int32(0)
    cost = C.c_float(0)
    sp = C.c_void_p(stream.cuda_stream) if stream is not None else None
    st = L.kpx_plan_static(C.byref(d), C.byref(w), C.byref(o), start.ctypes.data_as(C.POINTER(C.c_float)),
                           C.byref(g), C.byref(c), C.byref(cfg), int(n_iters), sp, int(capacity),
                           states.ctypes.data_as(C.POINTER(C.c_float)), controls.ctypes.data_as(C.POINTER(C.c_float)),
                           steps.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(ln), C.byref(cost))
    if st != KPX_OK:
        return int(st), None
    k = ln.value
    return int(st), dict(states=states[:k + 1], controls=controls[:k], steps=steps[:k], cost=float(cost.value))


def fp32_fma_rate(iters: int = 2048, stream=None) -> float:
    """kpx_fp32_fma_rate: the device's measured FP32 FMA throughput in
    TFLOP/s (one timed launch on `stream`, default the current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    st = load().kpx_fp32_fma_rate(int(iters), C.byref(out), C.c_void_p(s.cuda_stream))
    if st != KPX_OK:
        raise KpxError(st, "kpx_fp32_fma_rate")
    return float(out.value)


def last_create_error() -> str:
    """Message of the last failing kpx_create / kpx_plan_static in this thread."""
    return load().kpx_last_error(None).decode()


def status_str(s: int) -> str:
    return load().kpx_status_str(int(s)).decode()
