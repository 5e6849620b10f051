"""Host logic of the request loop (serve.py), on the CPU: the device arena
(admission by memory), per-class first-come-first-served admission, the
iteration budget, harvesting on a stopped planner, refusals of bad queries,
and the device-to-host clock mapping.  The batch is a fake with the
BatchPlanner interface, so faults are made on the host (a query whose
assignment raises, a planner that reports a full tree)."""
import types

import numpy as np
import pytest

from paper_2602_02846_gb300.serve import ALIGN, Arena, Request, Server, summarize

KPX_OK, KPX_TREE_FULL = 0, 4
INF = 0xFFFFFFFFFFFFFFFF


# -- arena ---------------------------------------------------------------------
def test_arena_first_fit_and_coalescing():
    a = Arena(10 * ALIGN + 17)
    assert a.capacity == 10 * ALIGN
    x = a.alloc(1)
    y = a.alloc(3 * ALIGN)
    z = a.alloc(2 * ALIGN + 1)
    assert (x, y, z) == (0, ALIGN, 4 * ALIGN)
    assert a.in_use == 7 * ALIGN and a.largest_free == 3 * ALIGN
    assert a.alloc(4 * ALIGN) is None
    a.free(y)
    assert a.alloc(2 * ALIGN) == ALIGN            # first fit reuses the hole
    a.free(x)
    a.free(ALIGN)
    a.free(z)
    assert a.in_use == 0 and a.largest_free == 10 * ALIGN   # everything merged back


def test_arena_random_against_byte_map():
    rng = np.random.default_rng(3)
    cap = 64 * ALIGN
    a = Arena(cap)
    owner = np.full(cap // ALIGN, -1)
    live = {}
    for step in range(3000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(len(live)))]
            a.free(off)
            owner[owner == off] = -1
            del live[off]
        else:
            n = int(rng.integers(1, 9 * ALIGN))
            off = a.alloc(n)
            units = (n + ALIGN - 1) // ALIGN
            free_runs = np.convolve((owner == -1).astype(int), np.ones(units, int), "valid")
            first = np.flatnonzero(free_runs == units)
            if off is None:
                assert first.size == 0
            else:
                assert off % ALIGN == 0 and off // ALIGN == first[0]   # first fit, exactly
                assert np.all(owner[off // ALIGN: off // ALIGN + units] == -1)
                owner[off // ALIGN: off // ALIGN + units] = off
                live[off] = units
        assert a.in_use == ALIGN * int(np.sum(owner != -1))


# -- a fake batch ----------------------------------------------------------------
class FakeMember:
    def __init__(self, slot):
        self.slot = slot

    def iterate(self, n, stats=False):
        s = self.slot
        return {"total_valid": 10 * s.iter, "status": s.status}

    def best_trajectory(self):
        return None if s_cost(self.slot) is None else {"cost": s_cost(self.slot)}


def s_cost(slot):
    p = slot.problem
    if p is None or p.solve_at is None or slot.iter < p.solve_at:
        return None
    return 10.0 - 0.01 * (slot.iter - p.solve_at)


class FakeBatch:
    """Slots advance one iteration per iterate() step while below their
    budget; device time is host time minus ``skew`` seconds."""

    def __init__(self, n_slots, clock, skew=5.0, iter_seconds=0.001, fail_rid=None):
        self.slots = [types.SimpleNamespace(problem=None, budget=0, iter=0, status=KPX_OK, vacant=True,
                                            t_start=0, t_first=0, t_last=0, bytes=0) for _ in range(n_slots)]
        self.clock, self.skew, self.iter_seconds = clock, skew, iter_seconds
        self.fail_rid = fail_rid
        self.max_bytes = 0
        self.assign_log = []

    def dev_ns(self):
        return int(round((self.clock.t - self.skew) * 1e9))

    def assign(self, i, prob, budget, workspace, offset, nbytes):
        if prob.rid == self.fail_rid:
            raise RuntimeError("invalid problem")
        s = self.slots[i]
        assert s.vacant, "slot reassigned while busy"
        s.problem, s.budget, s.iter, s.status, s.vacant = prob, budget, 0, KPX_OK, False
        s.t_start = s.t_first = s.t_last = 0
        s.bytes = nbytes
        self.assign_log.append((prob.rid, i, offset, nbytes))
        self.max_bytes = max(self.max_bytes, sum(x.bytes for x in self.slots if not x.vacant))

    def release(self, i):
        self.slots[i].vacant = True
        self.slots[i].bytes = 0

    def iterate(self, n):
        for _ in range(n):
            self.clock.t += self.iter_seconds
            for s in self.slots:
                if s.vacant or s.status != KPX_OK or s.iter >= s.budget:
                    continue
                if not s.t_start:
                    s.t_start = self.dev_ns()
                s.iter += 1
                if s.problem.full_at is not None and s.iter >= s.problem.full_at:
                    s.status = KPX_TREE_FULL
                if s_cost(s) is not None and not s.t_first:
                    s.t_first = self.dev_ns()
                s.t_last = self.dev_ns()

    def poll(self):
        out = []
        for s in self.slots:
            c = s_cost(s) if not s.vacant else None
            out.append({"status": -1 if s.vacant else s.status, "iter": s.iter, "n_nodes": s.iter,
                        "first_solution_iter": -1 if c is None else s.problem.solve_at,
                        "goal_cost": c, "t_start_ns": s.t_start, "t_first_solution_ns": s.t_first,
                        "t_last_ns": s.t_last, "t_poll_ns": self.dev_ns()})
        return out

    def member(self, i):
        return FakeMember(self.slots[i])


class FakeClock:
    def __init__(self):
        self.t = 100.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


def prob(rid, cls=0, nbytes=ALIGN, solve_at=None, full_at=None):
    return types.SimpleNamespace(rid=rid, dyn=cls, integ=0, name="fam%d" % cls, nbytes=nbytes,
                                 solve_at=solve_at, full_at=full_at)


def make_server(n_per_class, classes, arena_bytes, clock, **kw):
    slots, k = {}, 0
    for c in classes:
        slots[(c, 0)] = list(range(k, k + n_per_class))
        k += n_per_class
    batch = FakeBatch(k, clock, fail_rid=kw.pop("fail_rid", None))
    srv = Server(batch, slots, arena_bytes, iters_per_round=kw.pop("iters_per_round", 2),
                 workspace_size=lambda p: p.nbytes, clock=clock, sleep=clock.sleep, **kw)
    return srv, batch


def test_every_request_gets_its_budget_and_memory_is_returned():
    clock = FakeClock()
    srv, batch = make_server(3, [0, 1], 8 * ALIGN, clock)
    reqs = [Request(r, prob(r, cls=r % 2, nbytes=ALIGN * (1 + r % 3), solve_at=2), 0.001 * r, 5 + r % 4)
            for r in range(20)]
    out = srv.serve(reqs)
    assert all(o.status == "done" for o in out)
    for r, o in zip(reqs, out):
        assert o.iterations == r.iter_budget and o.cost == pytest.approx(10.0 - 0.01 * (r.iter_budget - 2))
        assert o.admitted >= o.arrival and o.finished >= o.admitted
    assert srv.arena.in_use == 0 and srv.arena.largest_free == 8 * ALIGN
    assert batch.max_bytes <= 8 * ALIGN          # admission by device memory
    assert all(s.vacant for s in batch.slots)


def test_memory_not_slots_limits_concurrency():
    clock = FakeClock()
    srv, batch = make_server(8, [0], 4 * ALIGN, clock)
    reqs = [Request(r, prob(r, nbytes=2 * ALIGN), 0.0, 4) for r in range(6)]
    out = srv.serve(reqs)
    # eight slots are free, but only two 2-unit queries fit the 4-unit arena at once
    assert batch.max_bytes == 4 * ALIGN
    assert all(off in (0, 2 * ALIGN) for _, _, off, _ in batch.assign_log)
    assert len(batch.assign_log) == 6 and all(o.status == "done" for o in out)
    assert sorted(o.admitted for o in out)[2] > 0.0   # the third waited for memory


def test_fifo_within_a_class():
    clock = FakeClock()
    srv, batch = make_server(1, [0, 1], 64 * ALIGN, clock)
    reqs = [Request(r, prob(r, cls=0 if r < 6 else 1), 0.0001 * r, 3) for r in range(9)]
    srv.serve(reqs)
    order0 = [rid for rid, *_ in batch.assign_log if rid < 6]
    assert order0 == sorted(order0)


def test_refusals_and_faults_are_contained():
    clock = FakeClock()
    srv, batch = make_server(2, [0], 4 * ALIGN, clock, fail_rid=3)
    reqs = [Request(0, prob(0, nbytes=5 * ALIGN), 0.0, 3),         # larger than the arena
            Request(1, prob(1, cls=7), 0.0, 3),                    # no slot of its class
            Request(2, prob(2, full_at=2, solve_at=1), 0.0, 9),    # its tree fills at iteration 2
            Request(3, prob(3), 0.0, 3),                           # assignment raises
            Request(4, prob(4, solve_at=1), 0.0, 4)]
    out = srv.serve(reqs)
    assert out[0].status.startswith("rejected") and "arena" in out[0].status
    assert out[1].status.startswith("rejected") and "class" in out[1].status
    assert out[2].status == "tree_full" and out[2].iterations == 2
    assert out[3].status.startswith("rejected") and "invalid" in out[3].status
    assert out[4].status == "done" and out[4].iterations == 4
    assert srv.arena.in_use == 0
    s = summarize(out, srv.offset, 1.0)
    assert s["rejected"] == 3 and s["served"] == 2


def test_realtime_arrivals_and_clock_mapping():
    clock = FakeClock()
    srv, batch = make_server(4, [0], 64 * ALIGN, clock, iters_per_round=1)
    reqs = [Request(r, prob(r, solve_at=3), 0.5 + 0.25 * r, 6) for r in range(4)]
    out = srv.serve(reqs, realtime=True)
    # device time = host time - 5 s; polls read the device clock with no
    # copy latency here, so the mapping is exact
    assert srv.offset == pytest.approx(5.0 - 100.0, abs=1e-9)
    for o in out:
        assert o.admitted >= o.arrival - 1e-12
        # the third iteration after admission finds the solution (1 ms each)
        assert o.ttfs() == pytest.approx(o.admitted - o.arrival + 0.003, abs=1e-6)
        assert o.cost_at(0.0025 + (o.admitted - o.arrival), srv.offset) is None
        assert o.cost_at(1.0, srv.offset) == pytest.approx(10.0 - 0.03)
