"""End-to-end parity in distribution: the CUDA planner and the FP64 oracle run
the same problems (seeds); their trees diverge after the first FP32/FP64
near-tie, so results are compared as distributions, with the bounds:

* success rates within a two-proportion 95 % bound (|p1 - p2| <= 1.96 se,
  se from the pooled rate, plus one problem of slack);
* median best costs within 5 % relative;
* Mann-Whitney U test of the best costs, p > 0.01;
* every GPU trajectory re-validated by the oracle in FP64 (segment error
  <= 1e-4, clearance >= -1e-4, goal reached within 1e-4, cost within 1e-4).

Seeds 0-99 of three families, one per system.  The quadcopter family is a
reduced configuration on both sides (120 boxes without walls, 2^15 nodes,
lambda 8, 20 iterations; the tree fills after about 14), so that 100 oracle
runs take a minute on the host cores.

The oracle runs in a process pool started (spawn) before the first GPU call.
"""
import concurrent.futures as cf
import math
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests import gpu_helpers as gh  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEEDS = list(range(100))

FAMILIES = {
    # the paper's large-delta DI setting scaled to a 32,768-node tree (16^3 x 2^3 regions)
    "di16": dict(kind="di", kw=dict(grid_pos=16, tree_cap=32768), iters=40),
    "dubins_open": dict(kind="dubins", kw=dict(n_obstacles=0, tree_cap=1 << 14, lam=16), iters=40),
    "quad_room": dict(kind="quad", kw=dict(clutter=120, certify=False, walls=False, tree_cap=1 << 15, lam=8),
                      iters=20),
}


def _make(kind, seed, kw):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2602_02846_gb300 import scenes
    return scenes.scene(kind, seed, **kw)


def _oracle_run(args):
    kind, seed, kw, iters = args
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    prob = _make(kind, seed, kw)
    pl = oracle.Planner(prob)
    pl.iterate(iters)
    tr = pl.best_trajectory()
    return seed, (tr["cost"] if tr else None)


@pytest.fixture(scope="module")
def oracle_results():
    ctx = mp.get_context("spawn")
    jobs = [(f["kind"], s, f["kw"], f["iters"]) for name, f in FAMILIES.items() for s in SEEDS]
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=ctx) as ex:
        out = list(ex.map(_oracle_run, jobs))
    res = {}
    i = 0
    for name in FAMILIES:
        res[name] = dict(out[i:i + len(SEEDS)])
        i += len(SEEDS)
    return res


@pytest.mark.parametrize("family", list(FAMILIES))
def test_success_and_cost_distributions_match_oracle(family, oracle_results):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as kpx
    from scipy import stats
    f = FAMILIES[family]
    gpu = {}
    worst_seg = 0.0
    for seed in SEEDS:
        prob = _make(f["kind"], seed, f["kw"])
        pl = kpx.Planner(prob)
        pl.iterate(f["iters"])
        tr = pl.best_trajectory()
        pl.close()
        gpu[seed] = tr["cost"] if tr else None
        if tr is not None:
            rv = gh.revalidate_trajectory(prob, tr)
            worst_seg = max(worst_seg, rv["max_seg_err"])
    orc = oracle_results[family]
    g_ok = [c for c in gpu.values() if c is not None]
    o_ok = [c for c in orc.values() if c is not None]
    n = len(SEEDS)
    p1, p2 = len(g_ok) / n, len(o_ok) / n
    pp = (len(g_ok) + len(o_ok)) / (2 * n)
    se = math.sqrt(max(pp * (1 - pp), 1e-12) * 2 / n)
    print(family, "success gpu %d/%d oracle %d/%d" % (len(g_ok), n, len(o_ok), n),
          "median cost gpu %.4f oracle %.4f" % (np.median(g_ok) if g_ok else -1, np.median(o_ok) if o_ok else -1),
          "worst segment error %.2e" % worst_seg)
    assert abs(p1 - p2) <= 1.96 * se + 1.0 / n
    assert len(g_ok) >= n // 2, "family should mostly succeed"
    mg, mo = float(np.median(g_ok)), float(np.median(o_ok))
    assert abs(mg - mo) <= 0.05 * mo
    p = stats.mannwhitneyu(g_ok, o_ok, alternative="two-sided").pvalue
    print(family, "Mann-Whitney p = %.3f" % p)
    assert p > 0.01
