"""Request loop with continuous batching.

Planning queries arrive over time.  A query is admitted when a slot of its
dynamics class is free and the device arena can hold its workspace
(kpx_workspace_size bytes: admission by device memory).  It is then planned
for an iteration budget that the device enforces (the slot stops iterating
once the budget is spent), and harvested when the budget is spent or its
planner stops (tree full).  All resident queries iterate in the same launches
(kpx_batch_iterate: one launch per phase for every slot), so a query that
arrives while others are on the GPU shares the device with them, and every
tree stays resident in HBM until it is harvested.

Each slot draws its controls from its own Philox key, and the batch kernels
keep each problem's work in its own slot order.  So a served query ends
bit-identical to the same problem planned alone with kpx_create for the same
number of iterations, whatever else was resident.

Time: the host clock (time.perf_counter, seconds from the start of serve())
is the reference.  Device events (first iteration, first solution) come as
%globaltimer stamps; each poll reads the device clock right before its copy
to the host, and the smallest (host - device) gap over all polls maps device
stamps onto the host clock (late by at most that poll's copy latency).
"""
from __future__ import annotations

import bisect
import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import scenes

ALIGN = 256


class Arena:
    """First-fit allocator over byte offsets [0, capacity) of one device
    buffer, in 256-byte units; freed ranges coalesce with their neighbours."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity) // ALIGN * ALIGN
        self._free: List[Tuple[int, int]] = [(0, self.capacity)] if self.capacity else []  # sorted (offset, size)
        self._used: Dict[int, int] = {}

    @staticmethod
    def rounded(nbytes: int) -> int:
        return (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN

    def alloc(self, nbytes: int) -> Optional[int]:
        size = self.rounded(nbytes)
        if size <= 0:
            size = ALIGN
        for i, (off, free) in enumerate(self._free):
            if free >= size:
                if free == size:
                    del self._free[i]
                else:
                    self._free[i] = (off + size, free - size)
                self._used[off] = size
                return off
        return None

    def free(self, off: int) -> None:
        size = self._used.pop(off)
        i = bisect.bisect_left(self._free, (off, 0))
        lo, hi = off, off + size
        if i < len(self._free) and self._free[i][0] == hi:      # merge the next range
            hi += self._free[i][1]
            del self._free[i]
        if i > 0 and self._free[i - 1][0] + self._free[i - 1][1] == lo:  # merge the previous one
            lo = self._free[i - 1][0]
            del self._free[i - 1]
            i -= 1
        self._free.insert(i, (lo, hi - lo))

    @property
    def in_use(self) -> int:
        return sum(self._used.values())

    @property
    def largest_free(self) -> int:
        return max((s for _, s in self._free), default=0)


@dataclasses.dataclass
class Request:
    rid: int
    problem: scenes.Problem
    arrival: float          # seconds after the start of serve()
    iter_budget: int        # iterations the device runs for it
    nbytes: int = 0         # device workspace (kpx_workspace_size), filled in by the server


@dataclasses.dataclass
class Outcome:
    rid: int
    family: str
    arrival: float
    admitted: Optional[float] = None
    finished: Optional[float] = None
    status: str = "waiting"             # "done", "tree_full", "rejected: ...", "error: ..."
    slot: int = -1
    nbytes: int = 0
    iterations: int = 0
    n_nodes: int = 0
    total_valid: int = 0
    cost: Optional[float] = None
    first_solution_iter: int = -1
    dev_start_ns: int = 0                # device clock stamps (0: none)
    dev_first_ns: int = 0
    trace: List[Tuple[int, Optional[float]]] = dataclasses.field(default_factory=list)  # (device ns, cost) per poll
    trajectory: Optional[dict] = None
    t_first: Optional[float] = None      # host clock of the first solution (set by finalize)

    def ttfs(self) -> Optional[float]:
        return None if self.t_first is None else self.t_first - self.arrival

    def cost_at(self, seconds_after_arrival: float, offset: float) -> Optional[float]:
        """Best cost the device had reported by ``seconds_after_arrival``
        (observed at poll granularity, so never optimistic)."""
        best = None
        for t_ns, c in self.trace:
            if t_ns * 1e-9 + offset - self.arrival <= seconds_after_arrival:
                best = c
        return best


class Server:
    """Continuous batching over one kpx batch.

    ``batch``: an object with assign(slot, problem, iter_limit, workspace,
    offset, nbytes), release(slot), iterate(n), poll(), member(slot)
    (BatchPlanner, or a fake of it for host-side tests); ``slots``: class key
    (dyn, integ) -> slot indices of that class; ``arena_tensor``: the device
    buffer the arena carves (None for a fake batch)."""

    def __init__(self, batch, slots: Dict[Tuple[int, int], Sequence[int]], arena_bytes: int,
                 arena_tensor=None, iters_per_round: int = 4, workspace_size: Optional[Callable] = None,
                 keep_trajectories: bool = True, on_finish: Optional[Callable] = None,
                 clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep):
        self.batch = batch
        self.free_slots = {k: collections.deque(v) for k, v in slots.items()}
        self.arena = Arena(arena_bytes)
        self.arena_tensor = arena_tensor
        self.iters_per_round = int(iters_per_round)
        if workspace_size is None:
            from . import kpx_workspace_size as workspace_size
        self.workspace_size = workspace_size
        self.keep_trajectories = keep_trajectories
        self.on_finish = on_finish
        self.clock, self.sleep = clock, sleep
        self.offset = None          # host seconds - device seconds (smallest gap seen)
        self.rounds = 0             # iterate + poll rounds
        self.resident_sum = 0       # resident queries summed over rounds
        self.admits = 0
        self.trajectories = 0

    @classmethod
    def create(cls, memory_bytes: int, slots_per_class: int = 32, families: Optional[Sequence] = None,
               device=None, stream=None, **kw) -> "Server":
        """A server on the GPU: ``slots_per_class`` slots for each dynamics
        class of ``families`` (template problems; default: the three families
        of the mixed workload) and an arena of ``memory_bytes`` device bytes
        for the queries' trees."""
        import torch
        from . import BatchPlanner
        if families is None:
            families = [scenes.di_scene(0, n_obstacles=0, tree_cap=256, grid_pos=16),
                        scenes.dubins_scene(0, n_obstacles=0, tree_cap=256),
                        scenes.quad_scene(0, clutter=0, certify=False, tree_cap=256)]
        templates, keys = [], []
        for f in families:
            for _ in range(slots_per_class):
                templates.append(f)
                keys.append((int(f.dyn), int(f.integ)))
        dev = torch.device(device if device is not None else "cuda")
        batch = BatchPlanner(templates, device=dev, stream=stream)
        for i in range(len(templates)):
            batch.release(i)
        slots: Dict[Tuple[int, int], List[int]] = {}
        for i, k in enumerate(keys):
            slots.setdefault(k, []).append(i)
        arena = torch.empty(int(memory_bytes) + ALIGN, dtype=torch.uint8, device=dev)
        return cls(batch, slots, int(memory_bytes), arena_tensor=arena, **kw)

    # -- one query ----------------------------------------------------------
    def _admit(self, req: Request, out: Outcome, now: float) -> bool:
        key = (int(req.problem.dyn), int(req.problem.integ))
        free = self.free_slots.get(key)
        if not free:
            return False
        off = self.arena.alloc(req.nbytes)
        if off is None:
            return False
        slot = free.popleft()
        try:
            if self.arena_tensor is not None:
                base = self.arena_tensor.data_ptr()
                pad = (-base) % ALIGN
                self.batch.assign(slot, req.problem, req.iter_budget, self.arena_tensor, pad + off, req.nbytes)
            else:
                self.batch.assign(slot, req.problem, req.iter_budget, None, off, req.nbytes)
        except Exception as e:  # invalid query: refuse it, keep serving
            self.arena.free(off)
            free.appendleft(slot)
            out.status = "rejected: %s" % e
            out.finished = now
            return True
        out.slot, out.nbytes, out.admitted, out.status = slot, req.nbytes, now, "running"
        self.admits += 1
        self._running[slot] = (req, out, off)
        return True

    def _harvest(self, slot: int, st: dict, now: float, tree_full: bool) -> None:
        req, out, off = self._running.pop(slot)
        m = self.batch.member(slot)
        if self.on_finish is not None:
            self.on_finish(req, out, m)
        stats = m.iterate(0, stats=True)
        out.total_valid = int(stats["total_valid"])
        out.iterations, out.n_nodes = int(st["iter"]), int(st["n_nodes"])
        out.cost = st["goal_cost"]
        out.first_solution_iter = int(st["first_solution_iter"])
        if self.keep_trajectories and out.cost is not None:
            out.trajectory = m.best_trajectory()
            self.trajectories += 1
        self.batch.release(slot)
        self.arena.free(off)
        self.free_slots[(int(req.problem.dyn), int(req.problem.integ))].append(slot)
        out.status = "tree_full" if tree_full else "done"
        out.finished = now

    # -- the loop -----------------------------------------------------------
    def serve(self, requests: Sequence[Request], realtime: bool = True) -> List[Outcome]:
        """Serves ``requests`` (arrival times relative to the call) to the end.
        realtime=False admits each query as soon as a slot and memory allow,
        ignoring arrival times (for tests)."""
        from . import KPX_OK, KPX_TREE_FULL
        reqs = sorted(requests, key=lambda r: r.arrival)
        outcomes = {r.rid: Outcome(r.rid, r.problem.name, r.arrival) for r in reqs}
        pending = collections.deque(reqs)
        waiting: Dict[Tuple[int, int], collections.deque] = collections.OrderedDict()
        self._running: Dict[int, Tuple[Request, Outcome, int]] = {}
        t0 = self.clock()
        clock = lambda: self.clock() - t0  # noqa: E731
        while pending or self._running or any(waiting.values()):
            now = clock()
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                if not r.nbytes:
                    r.nbytes = int(self.workspace_size(r.problem))
                o = outcomes[r.rid]
                if r.nbytes <= 0:
                    o.status, o.finished = "rejected: invalid problem", now
                elif r.nbytes > self.arena.capacity:
                    o.status, o.finished = "rejected: larger than the device arena", now
                elif (int(r.problem.dyn), int(r.problem.integ)) not in self.free_slots:
                    o.status, o.finished = "rejected: no slot of its dynamics class", now
                else:
                    waiting.setdefault((int(r.problem.dyn), int(r.problem.integ)), collections.deque()).append(r)
            # admission: per class, first come first served (a query that does
            # not fit yet holds back the later ones of its class)
            for q in waiting.values():
                while q and self._admit(q[0], outcomes[q[0].rid], now):
                    q.popleft()
            if not self._running:
                if pending and realtime:
                    self.sleep(max(0.0, pending[0].arrival - clock()))
                    continue
                if any(waiting.values()):
                    # nothing resident yet nothing admissible: the arena is
                    # fragmented beyond use or a class has no slots
                    for q in waiting.values():
                        while q:
                            r = q.popleft()
                            o = outcomes[r.rid]
                            o.status, o.finished = "rejected: could not be placed", clock()
                continue
            self.batch.iterate(self.iters_per_round)
            states = self.batch.poll()
            host_now = clock()
            self.rounds += 1
            self.resident_sum += len(self._running)
            t_poll = max(s["t_poll_ns"] for s in states)
            gap = host_now - t_poll * 1e-9
            self.offset = gap if self.offset is None else min(self.offset, gap)
            for slot in list(self._running):
                req, out, _ = self._running[slot]
                st = states[slot]
                if not out.dev_start_ns and st["t_start_ns"]:
                    out.dev_start_ns = st["t_start_ns"]
                if not out.dev_first_ns and st["t_first_solution_ns"]:
                    out.dev_first_ns = st["t_first_solution_ns"]
                out.trace.append((st["t_last_ns"], st["goal_cost"]))
                if st["status"] not in (KPX_OK,):
                    self._harvest(slot, st, host_now, st["status"] == KPX_TREE_FULL)
                    if st["status"] != KPX_TREE_FULL:
                        out.status = "error: status %d" % st["status"]
                elif st["iter"] >= req.iter_budget:
                    self._harvest(slot, st, host_now, False)
        off = self.offset if self.offset is not None else 0.0
        for o in outcomes.values():
            if o.dev_first_ns:
                o.t_first = o.dev_first_ns * 1e-9 + off
        return [outcomes[r.rid] for r in sorted(reqs, key=lambda r: r.rid)]


def summarize(outcomes: Sequence[Outcome], offset: float, wall: float, deadline: float = 0.1) -> dict:
    """p50/p99 time to first solution (from arrival), queueing delay,
    latency, cost at ``deadline`` seconds after arrival, throughput."""
    def pct(v, q):
        return float(np.percentile(v, q)) if v else None
    done = [o for o in outcomes if o.status in ("done", "tree_full")]
    ttfs = [o.ttfs() for o in done if o.ttfs() is not None]
    wait = [o.admitted - o.arrival for o in done]
    lat = [o.finished - o.arrival for o in done]
    c100 = [o.cost_at(deadline, offset) for o in done]
    c100 = [c for c in c100 if c is not None]
    final = [o.cost for o in done if o.cost is not None]
    by_family = {}
    for o in done:
        f = by_family.setdefault(o.family, {"served": 0, "solved": 0})
        f["served"] += 1
        f["solved"] += o.cost is not None
    return {
        "requests": len(outcomes), "served": len(done),
        "rejected": sum(o.status.startswith("rejected") for o in outcomes),
        "solved": sum(o.cost is not None for o in done),
        "ttfs_p50_ms": None if not ttfs else 1e3 * pct(ttfs, 50),
        "ttfs_p99_ms": None if not ttfs else 1e3 * pct(ttfs, 99),
        "wait_p50_ms": None if not wait else 1e3 * pct(wait, 50),
        "wait_p99_ms": None if not wait else 1e3 * pct(wait, 99),
        "latency_p50_ms": None if not lat else 1e3 * pct(lat, 50),
        "latency_p99_ms": None if not lat else 1e3 * pct(lat, 99),
        "cost_at_100ms_median": pct(c100, 50), "solved_by_100ms": len(c100),
        "final_cost_median": pct(final, 50),
        "requests_per_s": len(done) / wall if wall > 0 else None,
        "valid_per_s": sum(o.total_valid for o in done) / wall if wall > 0 else None,
        "families": by_family,
    }


def serve_plain(requests: Sequence[Request], device=None, stream=None, iters_per_round: int = 4,
                realtime: bool = True, clock: Callable[[], float] = time.perf_counter) -> List[Outcome]:
    """The same query stream through the plain planner, one query at a time
    in arrival order: kpx_create, kpx_iterate for its budget in rounds of
    ``iters_per_round`` (reading the best cost after each, as the server
    polls), best trajectory.  Trace times are host seconds (offset 0)."""
    import torch
    from . import KPX_OK, Planner
    dev = torch.device(device if device is not None else "cuda")
    reqs = sorted(requests, key=lambda r: r.arrival)
    outs = []
    t0 = clock()
    for r in reqs:
        now = clock() - t0
        if realtime and r.arrival > now:
            time.sleep(r.arrival - now)
        o = Outcome(r.rid, r.problem.name, r.arrival)
        o.admitted = clock() - t0
        pl = Planner(r.problem, device=dev, stream=stream)
        pl.stream.synchronize()
        t_begin = clock() - t0   # the GPU is idle: the first iteration starts now
        st = {"status": KPX_OK, "iter": 0}
        while st["status"] == KPX_OK and st["iter"] < r.iter_budget:
            st = pl.iterate(min(iters_per_round, r.iter_budget - st["iter"]), stats=True)
            cost = float(st["best_cost"])
            o.trace.append((int(round((clock() - t0) * 1e9)), cost if np.isfinite(cost) else None))
        o.finished = clock() - t0
        o.iterations, o.n_nodes, o.total_valid = int(st["iter"]), int(st["n_nodes"]), int(st["total_valid"])
        o.first_solution_iter = int(st["first_solution_iter"])
        if o.first_solution_iter >= 0:
            o.t_first = t_begin + st["first_solution_ns"] * 1e-9
        tr = pl.best_trajectory()
        o.cost = None if tr is None else float(tr["cost"])
        o.trajectory = tr
        o.status = "done" if st["status"] == KPX_OK else "tree_full"
        pl.close()
        outs.append(o)
    return sorted(outs, key=lambda o: o.rid)
