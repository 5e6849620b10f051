"""Adaptive delta on the GPU: kpx_set_regions remaps a live tree to a new
region grid exactly as the oracle's remap does (region ids, region keys,
dominated bits), and planning continues on the finer grid.  The literal
double-integrator configuration, which stalls on its 8^3 x 2^3 grid, grows
and solves after the grid is refined."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2602_02846_gb300 import scenes  # noqa: E402

SET_DOM, SET_ANC = 8, 4


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


def refined_axes(axes, factor=2, dims=(0, 1, 2)):
    return [scenes.RegionAxis(a.state_dim, a.bins * (factor if a.state_dim in dims else 1), a.lo, a.hi, a.wrap)
            for a in axes]


def _capacity(axes):
    return int(np.prod([a.bins for a in axes]))


CASES = {
    "di_literal": (lambda: scenes.di_scene(0), 30),
    "di16_growing": (lambda: scenes.di_scene(1, grid_pos=16, tree_cap=32768), 12),
    "dubins_forest": (lambda: scenes.dubins_scene(0), 20),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_remap_matches_oracle(kpx, case):
    make, iters = CASES[case]
    prob = make()
    fine = refined_axes(prob.axes)
    prob = dataclasses.replace(prob, region_capacity=_capacity(fine))
    pl = kpx.Planner(prob)
    pl.iterate(iters)
    before = pl.arrays()
    nn = before["n_nodes"]
    pl.set_regions(fine)
    after = pl.arrays()
    ref = oracle.remap_regions(dataclasses.replace(prob, axes=fine), before["x"].astype(np.float64),
                               before["key"], before["set"])
    assert np.array_equal(after["region"], ref["region"])
    R = _capacity(fine)
    assert np.array_equal(after["region_key"][:R], ref["region_key"])
    live = before["set"] != 3
    dom = (after["set_raw"] & SET_DOM) != 0
    assert np.array_equal(dom[live], ref["dominated"][live])
    assert not np.any(after["set_raw"][live] & SET_ANC)
    assert np.array_equal(after["set"], before["set"])  # sets are left to PruneNodes
    assert not ref["dominated"].any()  # a nested refinement dominates nobody
    # planning continues: the fused and the phase-kernel paths agree on the finer grid
    a = kpx.Planner(prob)
    b = kpx.Planner(prob, flags=kpx.KPX_FLAG_NO_FUSED)
    for p in (a, b):
        p.iterate(iters)
        p.set_regions(fine)
        p.iterate(7)
    sa, sb = a.arrays(), b.arrays()
    for k in ("x", "key", "parent", "region", "set_raw", "VA"):
        assert np.array_equal(np.ascontiguousarray(sa[k]).view(np.uint8), np.ascontiguousarray(sb[k]).view(np.uint8)), k
    assert sa["n_nodes"] >= nn
    for p in (pl, a, b):
        p.close()


def test_refining_the_stalled_di_configuration(kpx):
    prob = scenes.di_scene(0)  # 8^3 x 2^3 regions: stalls (a documented reading)
    fine = refined_axes(prob.axes)
    prob = dataclasses.replace(prob, region_capacity=_capacity(fine))
    pl = kpx.Planner(prob)
    st = pl.iterate(40, stats=True)
    stalled_nodes = st["n_nodes"]
    assert st["first_solution_iter"] < 0
    pl.set_regions(fine)
    st = pl.iterate(40, stats=True)
    assert st["n_nodes"] > 4 * stalled_nodes
    assert st["first_solution_iter"] >= 40, st
    tr = pl.best_trajectory()
    assert tr is not None
    # the solution re-validated in FP64 by the oracle
    rv = oracle.revalidate(prob, tr["states"].astype(np.float64), tr["controls"], tr["steps"])
    assert rv["ok"] and rv["max_seg_err"] < 1e-4, rv
    print("adaptive delta: stalled at %d nodes on 8^3 x 2^3; after refining to 16^3 x 2^3: %d nodes, "
          "first solution at iteration %d, cost %.4f" % (stalled_nodes, st["n_nodes"], st["first_solution_iter"],
                                                           tr["cost"]))
    pl.close()
