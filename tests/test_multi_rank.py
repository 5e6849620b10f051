"""Multi-process paths on CPU (gloo, world size 2).

1. The benchmark's replica reduction: every rank plans its own problem; the
   job value is the sum of valid rollouts over the max time over ranks.
2. The exchange that sharding one problem would need: ranks split the slots
   of an iteration, propagate their shard, all-reduce MIN the region keys and
   all-gather their winners; the result must be bit-identical to the
   unsharded step.  Run with the FP64 oracle as the per-rank engine.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

INF = 0xFFFFFFFFFFFFFFFF
SIGN = np.uint64(1 << 63)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _replica_worker(rank, world, port, q):
    _init(rank, world, port)
    import bench
    valid = 1000 * (rank + 1)
    ms = 10.0 + 5.0 * rank
    tot = bench.allreduce(valid, "sum", torch.device("cpu"))
    mx = bench.allreduce(ms, "max", torch.device("cpu"))
    bench.barrier()
    q.put((rank, tot, mx))
    dist.destroy_process_group()


def test_replica_reduction_gloo():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, mx in out:
        assert tot == 3000.0 and mx == 15.0


def _to_signed(keys):
    """Order-preserving map of uint64 keys (all below 2^63 except INF) to int64."""
    k = np.asarray(keys, np.uint64)
    return np.where(k == np.uint64(INF), np.iinfo(np.int64).max, k.astype(np.int64))


def _from_signed(v):
    v = np.asarray(v, np.int64)
    return np.where(v == np.iinfo(np.int64).max, np.uint64(INF), v.astype(np.uint64))


def _shard_worker(rank, world, port, q):
    _init(rank, world, port)
    import oracle
    from paper_2602_02846_gb300 import scenes
    prob = scenes.di_scene(1, grid_pos=16, tree_cap=32768)
    pl = oracle.Planner(prob)
    pl.iterate(3)  # identical on every rank
    st = pl.state()
    n_slots = st["count_A"] * prob.lam
    lo = n_slots * rank // world
    hi = n_slots * (rank + 1) // world
    slots = np.arange(lo, hi, dtype=np.int64)
    rec = oracle.propagate(prob, st["iter"], prob.lam, st["x"], st["cost"], st["VA"], st["count_A"], slots=slots)
    # local region minimum over this shard's valid candidates
    rk_local = st["region_key"].copy()
    for i in np.nonzero(rec["valid"])[0]:
        r = rec["region"][i]
        rk_local[r] = min(rk_local[r], rec["key"][i])
    t = torch.from_numpy(_to_signed(rk_local))
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    rk_global = _from_signed(t.numpy())
    # local winners: candidates still holding their region's global key
    mine = [int(rec["slot"][i]) for i in np.nonzero(rec["valid"])[0]
            if rec["key"][i] == rk_global[rec["region"][i]]]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    winners = sorted(s for part in gathered for s in part)
    # unsharded reference on rank 0
    ref = None
    if rank == 0:
        full = oracle.propagate(prob, st["iter"], prob.lam, st["x"], st["cost"], st["VA"], st["count_A"])
        rk_ref, win, kept, full_flag = oracle.select_winners(st["region_key"], st["region_key"], full["valid"],
                                                             full["region"], full["key"], st["n_nodes"],
                                                             prob.tree_cap)
        ref = (rk_ref.tolist(), [int(full["slot"][w]) for w in win])
    q.put((rank, rk_global.tolist(), winners, ref))
    dist.destroy_process_group()


def test_sharded_iteration_exchange_matches_unsharded():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, rk, win, ref = q.get(timeout=300)
        out[rank] = (rk, win, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rk_ref, win_ref = out[0][2]
    for rank in (0, 1):
        assert out[rank][0] == rk_ref
        assert out[rank][1] == win_ref
    assert len(win_ref) > 0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "1")
    args = bench.parse_args(["--impl", "reference"])
    # rank != 0: returns immediately, prints nothing (no process group is needed)
    monkeypatch.setattr(bench, "dist_setup", lambda backend: (2, 1, 1))
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
