"""Trajectory refinement post-pass for the 12D quadcopter (optional; the
planner never calls it).

``RolloutObjective`` is a ``torch.autograd.Function`` over a batch of
control sequences.  Its forward is the kpx_refine_eval objective (effort +
duration, a softplus penalty on the signed distance to every box after each
RK4 step, and a goal pull; include/kpx.h).  Its backward is the hand-written
adjoint rollout with checkpoints.  ``refine`` runs projected Adam on the
controls, keeps each trajectory's best iterate, and re-validates the result
with the planner's own FP32 stepper and an FP64 cost sum
(kpx_refine_validate).  A trajectory keeps its refined controls only if they
are valid and lower its objective.  All arithmetic runs in the library's
kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import KPX_OK, KpxError, kpx_dynamics, kpx_goal, kpx_workspace, load, problem_structs

EXPORTED = ("kpx_refine_workspace_size", "kpx_refine_eval", "kpx_refine_validate", "kpx_refine_adam",
            "kpx_refine_keep_best")


class kpx_refine_cost(C.Structure):
    _fields_ = [("w_obs", C.c_float), ("beta", C.c_float), ("margin", C.c_float), ("w_goal", C.c_float),
                ("goal", C.c_float * 3), ("w_effort", C.c_float)]


_declared = False


def _lib():
    global _declared
    L = load()
    if not _declared:
        vp = C.c_void_p
        L.kpx_refine_workspace_size.argtypes = [C.c_int32, C.c_int32]
        L.kpx_refine_workspace_size.restype = C.c_size_t
        L.kpx_refine_eval.argtypes = [C.POINTER(kpx_dynamics), C.POINTER(kpx_refine_cost), vp, C.c_int32, C.c_int32,
                                      C.c_int32, vp, vp, vp, vp, vp, C.c_int32, vp, vp, vp, C.c_size_t, vp]
        L.kpx_refine_eval.restype = C.c_int
        L.kpx_refine_validate.argtypes = [C.POINTER(kpx_dynamics), C.POINTER(kpx_workspace), vp, C.c_int32,
                                          C.POINTER(kpx_goal), C.c_float, C.c_int32, C.c_int32, vp, vp, vp, vp,
                                          vp, vp, vp, vp]
        L.kpx_refine_validate.restype = C.c_int
        L.kpx_refine_adam.argtypes = [C.POINTER(kpx_dynamics), C.c_int32, C.c_int32, vp, vp, vp, vp, vp, C.c_int32,
                                      C.c_float, vp]
        L.kpx_refine_adam.restype = C.c_int
        L.kpx_refine_keep_best.argtypes = [C.c_int32, C.c_int32, vp, vp, vp, vp, vp]
        L.kpx_refine_keep_best.restype = C.c_int
        _declared = True
    return L


def default_cost(prob, w_obs: float = 1.0, beta: float = 200.0, margin: float = 0.01, w_goal: float = 10.0) -> dict:
    """Objective weights for a problem: its goal centre and effort weight."""
    return dict(w_obs=w_obs, beta=beta, margin=margin, w_goal=w_goal, goal=list(prob.goal_c),
                w_effort=float(prob.w_effort))


def _cost_struct(spec) -> kpx_refine_cost:
    c = kpx_refine_cost()
    c.w_obs, c.beta, c.margin, c.w_goal = spec["w_obs"], spec["beta"], spec["margin"], spec["w_goal"]
    for a in range(3):
        c.goal[a] = spec["goal"][a]
    c.w_effort = spec["w_effort"]
    return c


def _check(st, what):
    if st != KPX_OK:
        raise KpxError(st, what)


class Batch:
    """A batch of control sequences on the device: u[B][S][4] float32,
    steps[B][S] int32, n_seg[B] int32, x0[B][12] float32, obstacles[M][6]."""

    def __init__(self, prob, x0, u, steps, n_seg, obstacles=None, device=None):
        import torch
        dev = torch.device(device if device is not None else "cuda")
        self.prob = prob
        self.x0 = torch.as_tensor(np.asarray(x0, np.float32), device=dev).contiguous()
        self.u = torch.as_tensor(np.asarray(u, np.float32), device=dev).contiguous()
        self.steps = torch.as_tensor(np.asarray(steps, np.int32), device=dev).contiguous()
        self.n_seg = torch.as_tensor(np.asarray(n_seg, np.int32), device=dev).contiguous()
        obs = prob.obstacles if obstacles is None else obstacles
        self.obs = torch.as_tensor(np.asarray(obs, np.float32).reshape(-1, 6), device=dev).contiguous()
        self.count, self.max_segments = int(self.u.shape[0]), int(self.u.shape[1])
        st = np.asarray(steps, np.int64)
        ns = np.asarray(n_seg, np.int64)
        mask = np.arange(st.shape[1])[None, :] < ns[:, None]
        totals = (st * mask).sum(1)
        self.max_total_steps = int(totals.max()) if self.count else 0
        # longest first: the launch takes trajectories in this order
        order = np.argsort(-totals, kind="stable").astype(np.int32)
        self.order = torch.as_tensor(order, device=dev).contiguous()
        d, w, o, g, c, cfg, obsa, start = problem_structs(prob)
        self._structs = (d, w, g)
        self.dyn, self.ws, self.goal = d, w, g

    @classmethod
    def from_trajectories(cls, prob, trajs: Sequence[dict], device=None, max_segments: Optional[int] = None):
        """From planner trajectories (dicts of states, controls, steps)."""
        B = len(trajs)
        S = max_segments or max(len(t["steps"]) for t in trajs)
        u = np.zeros((B, S, 4), np.float32)
        steps = np.zeros((B, S), np.int32)
        x0 = np.zeros((B, 12), np.float32)
        n_seg = np.zeros(B, np.int32)
        for i, t in enumerate(trajs):
            k = len(t["steps"])
            u[i, :k] = t["controls"]
            steps[i, :k] = t["steps"]
            x0[i] = t["states"][0]
            n_seg[i] = k
        return cls(prob, x0, u, steps, n_seg, device=device)


def evaluate(batch: Batch, spec, u=None, grad: bool = False, stream=None):
    """Objective J[B] (and dJ/du when grad) for the batch's controls (or u)."""
    import torch
    L = _lib()
    u = batch.u if u is None else u
    J = torch.empty(batch.count, dtype=torch.float32, device=u.device)
    g = torch.empty_like(u) if grad else None
    # the workspace: the box grid, plus the checkpoints for a gradient; the
    # same grid either way, so J is the same with and without a gradient
    size = int(L.kpx_refine_workspace_size(batch.count, batch.max_total_steps) if grad
               else L.kpx_refine_workspace_size(0, 0))
    ws = torch.empty(size + 256, dtype=torch.uint8, device=u.device)
    s = stream if stream is not None else torch.cuda.current_stream(u.device)
    cost = _cost_struct(spec)
    wptr = ws.data_ptr() + ((-ws.data_ptr()) % 256)
    _check(L.kpx_refine_eval(C.byref(batch.dyn), C.byref(cost), C.c_void_p(batch.obs.data_ptr()),
                             int(batch.obs.shape[0]), batch.count, batch.max_segments,
                             C.c_void_p(batch.x0.data_ptr()), C.c_void_p(u.data_ptr()),
                             C.c_void_p(batch.steps.data_ptr()), C.c_void_p(batch.n_seg.data_ptr()),
                             C.c_void_p(batch.order.data_ptr()), batch.max_total_steps, C.c_void_p(J.data_ptr()),
                             C.c_void_p(g.data_ptr()) if grad else None, C.c_void_p(wptr), C.c_size_t(size),
                             C.c_void_p(s.cuda_stream)), "kpx_refine_eval")
    batch.last_workspace = (ws, wptr)  # kept for box_tests()
    return (J, g) if grad else J


def box_tests(batch: Batch, stream=None):
    """The box tests of the batch's last evaluate (kpx_refine_counters):
    (objective candidates, objective terms, gradient candidates, gradient
    terms).  Synchronises the stream."""
    import torch
    if getattr(batch, "last_workspace", None) is None:
        raise RuntimeError("box_tests: no evaluate() on this batch yet")
    ws, wptr = batch.last_workspace
    s = stream if stream is not None else torch.cuda.current_stream(ws.device)
    out = (C.c_uint64 * 4)()
    _check(_lib().kpx_refine_counters(C.c_void_p(wptr), out, C.c_void_p(s.cuda_stream)), "kpx_refine_counters")
    return tuple(int(v) for v in out)


def validate(batch: Batch, u=None, stream=None):
    """(valid[B] bool, cost[B] float64 (FP64 sum of the edge costs), x_end[B][12])."""
    import torch
    L = _lib()
    u = batch.u if u is None else u
    valid = torch.empty(batch.count, dtype=torch.int32, device=u.device)
    cost = torch.empty(batch.count, dtype=torch.float64, device=u.device)
    xe = torch.empty((batch.count, 12), dtype=torch.float32, device=u.device)
    s = stream if stream is not None else torch.cuda.current_stream(u.device)
    _check(L.kpx_refine_validate(C.byref(batch.dyn), C.byref(batch.ws), C.c_void_p(batch.obs.data_ptr()),
                                 int(batch.obs.shape[0]), C.byref(batch.goal), float(batch.prob.w_effort),
                                 batch.count, batch.max_segments, C.c_void_p(batch.x0.data_ptr()),
                                 C.c_void_p(u.data_ptr()), C.c_void_p(batch.steps.data_ptr()),
                                 C.c_void_p(batch.n_seg.data_ptr()), C.c_void_p(valid.data_ptr()),
                                 C.c_void_p(cost.data_ptr()), C.c_void_p(xe.data_ptr()), C.c_void_p(s.cuda_stream)),
           "kpx_refine_validate")
    return valid.bool(), cost, xe


def _autograd_function():
    import torch

    class RolloutObjective(torch.autograd.Function):
        """J = objective(u) per trajectory; backward = the adjoint kernel."""

        @staticmethod
        def forward(ctx, u, batch, spec):
            ctx.batch, ctx.spec = batch, spec
            ctx.save_for_backward(u)
            return evaluate(batch, spec, u=u.detach().contiguous())

        @staticmethod
        def backward(ctx, gJ):
            (u,) = ctx.saved_tensors
            _, g = evaluate(ctx.batch, ctx.spec, u=u.detach().contiguous(), grad=True)
            return gJ.reshape(-1, 1, 1).to(g.dtype) * g, None, None

    return RolloutObjective


_fn = None


def objective(u, batch: Batch, spec):
    """Differentiable objective: J[B] = RolloutObjective.apply(u, batch, spec)."""
    global _fn
    if _fn is None:
        _fn = _autograd_function()
    return _fn.apply(u, batch, spec)


def refine(batch: Batch, spec, iters: int = 40, lr: float = 0.02, stream=None):
    """Projected Adam on the controls (scaled to [-1, 1] by the control
    box); the best iterate of each trajectory is kept, then re-validated.
    Returns dict(u, J0, J, valid, cost0, cost, accepted): a trajectory is
    accepted (its refined controls returned) when the refined sequence is
    valid and its objective is lower; otherwise its original controls stay."""
    import torch
    L = _lib()
    s = stream if stream is not None else torch.cuda.current_stream(batch.u.device)
    sp = C.c_void_p(s.cuda_stream)
    u = batch.u.clone()
    J0 = evaluate(batch, spec, u=u, stream=s)
    u_best, J_best = u.clone(), J0.clone()
    m1, m2 = torch.zeros_like(u), torch.zeros_like(u)
    for t in range(1, iters + 1):
        J, g = evaluate(batch, spec, u=u, grad=True, stream=s)
        _check(L.kpx_refine_keep_best(batch.count, batch.max_segments, C.c_void_p(u.data_ptr()),
                                      C.c_void_p(J.data_ptr()), C.c_void_p(u_best.data_ptr()),
                                      C.c_void_p(J_best.data_ptr()), sp), "kpx_refine_keep_best")
        _check(L.kpx_refine_adam(C.byref(batch.dyn), batch.count, batch.max_segments,
                                 C.c_void_p(batch.n_seg.data_ptr()), C.c_void_p(u.data_ptr()),
                                 C.c_void_p(g.data_ptr()), C.c_void_p(m1.data_ptr()), C.c_void_p(m2.data_ptr()), t,
                                 float(lr), sp), "kpx_refine_adam")
    J = evaluate(batch, spec, u=u, stream=s)
    _check(L.kpx_refine_keep_best(batch.count, batch.max_segments, C.c_void_p(u.data_ptr()), C.c_void_p(J.data_ptr()),
                                  C.c_void_p(u_best.data_ptr()), C.c_void_p(J_best.data_ptr()), sp),
           "kpx_refine_keep_best")
    valid0, cost0, _ = validate(batch, u=batch.u, stream=s)
    valid, cost, _ = validate(batch, u=u_best, stream=s)
    accepted = valid & (J_best < J0)
    out_u = torch.where(accepted.reshape(-1, 1, 1), u_best, batch.u)
    return dict(u=out_u, J0=J0, J=torch.where(accepted, J_best, J0), valid0=valid0, valid=valid, cost0=cost0,
                cost=torch.where(accepted, cost, cost0), accepted=accepted)
