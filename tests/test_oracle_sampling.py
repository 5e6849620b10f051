"""Oracle pins: Philox4x32-10 and the control/duration sampling of Alg. 2.

Pins: the published known-answer vectors (tests/golden), the wiring of
Philox words to controls checked by hand against those vectors, and the
distributional properties the sampling must have (uniform u on [lo, hi],
uniform K on [k_min, k_max], distinct counters give distinct draws).
"""
import math
import os

import numpy as np
import pytest

from paper_2602_02846_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = oracle_mod.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == out


def test_philox_words_are_uniform(oracle_mod):
    # chi-square over 16 bins of the top 4 bits of 4 * 4096 words
    counts = np.zeros(16)
    for i in range(4096):
        w = oracle_mod.philox4x32_10([i, 7, 0, 0], [1234, 0])
        for x in w:
            counts[int(x) >> 28] += 1
    exp = counts.sum() / 16
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 37.7  # 15 dof, p = 0.001


def test_sample_wiring_against_kat(oracle_mod):
    """seed 0, (iter, node, sample) = (0, 0, 0) draws the first KAT vector:
    u_i from words 0..m-1 via f = (w >> 8) / 2^24, K from word m."""
    p = scenes.di_scene(0, planner_seed=0)
    u, K = oracle_mod.sample_control(p, 0, 0, 0)
    words = [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    for i in range(3):
        f = np.float32((words[i] >> 8) / 2.0 ** 24)
        # lo = -1, hi = 1: u = -1 + 2 f (each step exact in FP32 here)
        assert u[i] == np.float32(-1.0) + np.float32(2.0) * f
    assert K == 5 + (words[3] * 26 >> 32)
    # quadcopter (m = 4): K comes from word 0 of the second block
    q = scenes.quad_scene(0, clutter=0, certify=False, planner_seed=0)
    uq, Kq = oracle_mod.sample_control(q, 0, 0, 0)
    w1 = oracle_mod.philox4x32_10([0, 0, 0, 1], [0, 0])
    assert Kq == 10 + (int(w1[0]) * 51 >> 32)
    span = np.float32(q.u_hi[0]) - np.float32(q.u_lo[0])
    f0 = np.float32((words[0] >> 8) / 2.0 ** 24)
    assert uq[0] == np.float32(q.u_lo[0]) + np.float32(span * f0)


def test_seed_words_and_counter_fields(oracle_mod):
    """The 64-bit seed is split into (low, high) key words; iteration, node
    and sample occupy counter words 0, 1, 2."""
    p = scenes.di_scene(0, planner_seed=(7 << 32) | 5)
    u, K = oracle_mod.sample_control(p, 3, 11, 2)
    w = oracle_mod.philox4x32_10([3, 11, 2, 0], [5, 7])
    assert u[0] == np.float32(-1.0) + np.float32(2.0) * np.float32((int(w[0]) >> 8) / 2.0 ** 24)
    assert K == 5 + (int(w[3]) * 26 >> 32)


def test_sample_distribution(oracle_mod):
    p = scenes.dubins_scene(0, n_obstacles=0)
    us, ks = [], []
    for node in range(64):
        for s in range(64):
            u, K = oracle_mod.sample_control(p, 1, node, s)
            us.append(u)
            ks.append(K)
    us = np.array(us)
    ks = np.array(ks)
    for i in range(3):
        assert us[:, i].min() >= p.u_lo[i] and us[:, i].max() <= p.u_hi[i]
        # mean of U[lo,hi] within 4 sigma
        mu = (p.u_lo[i] + p.u_hi[i]) / 2
        sd = (p.u_hi[i] - p.u_lo[i]) / math.sqrt(12) / math.sqrt(len(us))
        assert abs(us[:, i].mean() - mu) < 4 * sd
    assert ks.min() == p.k_min and ks.max() == p.k_max
    counts = np.bincount(ks - p.k_min, minlength=p.k_max - p.k_min + 1)
    exp = len(ks) / counts.size
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 49.7  # 20 dof, p = 0.001
    # distinct counters -> distinct draws
    assert len({tuple(np.round(r, 7)) for r in us}) == len(us)
