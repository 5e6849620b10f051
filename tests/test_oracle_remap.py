"""Pins of the oracle's region remap (adaptive delta): a hand example, and
the refinement invariant on whole oracle runs (a finer nested grid leaves
no non-terminal node dominated, one non-terminal node per non-empty
region)."""
import dataclasses

import numpy as np

from paper_2602_02846_gb300 import scenes

INF = 0xFFFFFFFFFFFFFFFF


def test_remap_hand_example(oracle_mod):
    base = scenes.di_scene(0, n_obstacles=0)
    prob = dataclasses.replace(base, axes=[scenes.RegionAxis(0, 4, 0.0, 1.0)])
    x = np.zeros((5, 6))
    x[:, 0] = [0.1, 0.2, 0.3, 0.6, 0.9]
    key = np.array([(5 << 32) | 0, (3 << 32) | 1, (1 << 32) | 2, (2 << 32) | 3, (7 << 32) | 4], np.uint64)
    sets = np.array([1, 2, 3, 1, 1], np.uint8)  # A, I, T, A, A
    r = oracle_mod.remap_regions(prob, x, key, sets)
    assert list(r["region"]) == [0, 0, 1, 2, 3]
    # region 1 holds only a terminal node: empty
    assert [int(v) for v in r["region_key"]] == [int(key[1]), INF, int(key[3]), int(key[4])]
    assert list(r["dominated"]) == [True, False, False, False, False]


def _refined(prob, factor):
    axes = [scenes.RegionAxis(a.state_dim, a.bins * (factor if a.state_dim < 3 else 1), a.lo, a.hi, a.wrap)
            for a in prob.axes]
    return dataclasses.replace(prob, axes=axes)


def test_refinement_invariant_on_oracle_runs(oracle_mod):
    for prob, iters in [(scenes.di_scene(1, grid_pos=8, tree_cap=4096), 25),
                        (scenes.dubins_scene(2, n_obstacles=40, tree_cap=4096, lam=8), 12)]:
        pl = oracle_mod.Planner(prob)
        pl.iterate(iters)
        st = pl.state()
        nn = st["n_nodes"]
        x, key, sets = st["x"][:nn], st["key"][:nn], st["set"][:nn]
        # the same grid: the oracle's own region keys, no dominated non-terminal node
        same = oracle_mod.remap_regions(prob, x, key, sets)
        assert np.array_equal(same["region"], st["region"][:nn])
        assert not same["dominated"].any()
        fine = oracle_mod.remap_regions(_refined(prob, 2), x, key, sets)
        assert not fine["dominated"].any()
        live = sets != 3
        regions = fine["region"][live]
        assert len(np.unique(regions)) == live.sum()  # one non-terminal node per region
        assert np.array_equal(fine["region_key"][regions], key[live])
