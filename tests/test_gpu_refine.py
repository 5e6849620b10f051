"""The refinement post-pass on the GPU against the FP64 oracle: the objective
and its adjoint gradient (FP32 vs FP64, stated errors), central differences
of the GPU objective (eps = 1e-3 in control units scaled to [-1, 1]), long
horizons through the checkpoints, the torch.autograd.Function, the FP32
re-validation kernel, and refinement of trajectories returned by the planner
(re-validated by the oracle in FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2602_02846_gb300 import scenes  # noqa: E402


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


@pytest.fixture(scope="module")
def rf(kpx):
    from paper_2602_02846_gb300 import refine
    return refine


def _case(B, S_range, K_range, n_boxes, seed, speed=0.8):
    """Controls near hover from a start moving along +x, with boxes scattered
    near the flight line so that the penalty is active."""
    prob = scenes.quad_scene(0, clutter=-1)
    rng = np.random.default_rng(seed)
    S = S_range[1]
    mg = float(prob.param[0]) * float(prob.param[1])
    n_seg = rng.integers(S_range[0], S_range[1] + 1, B).astype(np.int32)
    steps = rng.integers(K_range[0], K_range[1] + 1, (B, S)).astype(np.int32)
    u = np.zeros((B, S, 4), np.float32)
    u[:, :, 0] = mg + rng.uniform(-0.8, 0.8, (B, S))
    u[:, :, 1:] = rng.uniform(-0.004, 0.004, (B, S, 3))
    mask = np.arange(S)[None, :] < n_seg[:, None]
    u *= mask[:, :, None]
    steps *= mask
    x0 = np.tile(np.asarray(prob.start, np.float32), (B, 1))
    x0[:, 6] = speed
    c = np.column_stack([rng.uniform(0.1, 0.9, n_boxes), 0.5 + rng.uniform(-0.05, 0.05, (n_boxes, 2))])
    e = rng.uniform(0.004, 0.015, (n_boxes, 3))
    c[:, 1] += np.where(rng.uniform(-1, 1, n_boxes) > 0, 1, -1) * (0.03 + e[:, 1])
    obs = np.concatenate([c - e, c + e], 1).astype(np.float32)
    return prob, x0, u, steps, n_seg, obs


SPEC = dict(w_obs=1.0, beta=200.0, margin=0.01, w_goal=10.0, goal=[0.95, 0.5, 0.5], w_effort=1.0)


def _oracle_grad(prob, x0, u, steps, n, obs):
    return oracle.refine_grad(prob, SPEC, x0.astype(np.float64), u[:n].astype(np.float64), steps[:n],
                              obstacles=obs.astype(np.float64))


def test_objective_and_gradient_match_fp64_oracle(rf):
    prob, x0, u, steps, n_seg, obs = _case(6, (8, 40), (10, 60), 60, seed=1)
    batch = rf.Batch(prob, x0, u, steps, n_seg, obstacles=obs)
    J, g = rf.evaluate(batch, SPEC, grad=True)
    J, g = J.cpu().numpy(), g.cpu().numpy()
    errs = []
    for i in range(6):
        n = int(n_seg[i])
        J64, g64 = _oracle_grad(prob, x0[i], u[i], steps[i], n, obs)
        assert abs(J[i] - J64) <= 1e-4 * abs(J64), (i, J[i], J64)
        rel = np.abs(g[i, :n] - g64).max() / np.abs(g64).max()
        errs.append(rel)
        assert rel < 2e-3, (i, rel)
        assert np.all(g[i, n:] == 0.0)
    print("FP32 adjoint vs FP64 gradient, worst relative (max-norm):", max(errs))


def test_gradient_matches_central_differences(rf):
    prob, x0, u, steps, n_seg, obs = _case(2, (6, 10), (10, 40), 40, seed=2)
    batch = rf.Batch(prob, x0, u, steps, n_seg, obstacles=obs)
    _, g = rf.evaluate(batch, SPEC, grad=True)
    g = g.cpu().numpy()
    half = 0.5 * (np.asarray(prob.u_hi[:4], np.float64) - np.asarray(prob.u_lo[:4], np.float64))
    rng = np.random.default_rng(0)
    worst = 0.0
    for i in range(2):
        n = int(n_seg[i])
        # the gradient in scaled coordinates z = (u - mid) / half, against
        # central differences of the GPU objective with eps = 1e-3 in z
        coords = [(int(rng.integers(n)), c) for c in range(4) for _ in range(3)]
        gz = np.array([g[i, s, c] * half[c] for s, c in coords])
        fd = []
        for s, c in coords:
            up, um = u.copy(), u.copy()
            up[i, s, c] += np.float32(1e-3 * half[c])
            um[i, s, c] -= np.float32(1e-3 * half[c])
            dz = (float(up[i, s, c]) - float(um[i, s, c])) / half[c]  # the FP32-rounded step
            Jp = rf.evaluate(batch, SPEC, u=torch.as_tensor(up, device="cuda"))[i].item()
            Jm = rf.evaluate(batch, SPEC, u=torch.as_tensor(um, device="cuda"))[i].item()
            fd.append((Jp - Jm) / dz)
        fd = np.array(fd)
        rel = np.abs(gz - fd).max() / np.abs(fd).max()
        worst = max(worst, rel)
        assert rel < 2e-2, (i, rel, gz, fd)
    print("adjoint vs central differences (eps 1e-3, scaled), worst relative:", worst)


def test_long_horizon_through_checkpoints(rf):
    """512 segments (about 15,000 RK4 steps, 470 checkpoint intervals)."""
    prob, x0, u, steps, n_seg, obs = _case(2, (512, 512), (20, 40), 30, seed=3, speed=0.05)
    batch = rf.Batch(prob, x0, u, steps, n_seg, obstacles=obs)
    J, g = rf.evaluate(batch, SPEC, grad=True)
    J, g = J.cpu().numpy(), g.cpu().numpy()
    for i in range(2):
        J64, g64 = _oracle_grad(prob, x0[i], u[i], steps[i], 512, obs)
        assert abs(J[i] - J64) <= 1e-3 * abs(J64), (i, J[i], J64)
        rel = np.abs(g[i] - g64).max() / np.abs(g64).max()
        print("long horizon: FP32 adjoint vs FP64 gradient, relative (max-norm):", rel)
        assert rel < 1e-2, rel


def test_autograd_function(rf):
    prob, x0, u, steps, n_seg, obs = _case(4, (5, 12), (10, 30), 20, seed=4)
    batch = rf.Batch(prob, x0, u, steps, n_seg, obstacles=obs)
    ut = batch.u.clone().requires_grad_(True)
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], device="cuda")
    J = rf.objective(ut, batch, SPEC)
    (w * J).sum().backward()
    _, g = rf.evaluate(batch, SPEC, grad=True)
    assert torch.equal(ut.grad, w.reshape(-1, 1, 1) * g)
    assert torch.equal(J.detach(), rf.evaluate(batch, SPEC))


def test_validate_matches_fp64_oracle(rf):
    prob, x0, u, steps, n_seg, obs = _case(16, (3, 12), (10, 40), 40, seed=5, speed=0.3)
    prob.obstacles = obs
    batch = rf.Batch(prob, x0, u, steps, n_seg)
    valid, cost, xe = rf.validate(batch)
    valid, cost = valid.cpu().numpy(), cost.cpu().numpy()
    agree = 0
    for i in range(16):
        n = int(n_seg[i])
        r = oracle.validate_controls(prob, x0[i].astype(np.float64), u[i, :n], steps[i, :n])
        assert abs(cost[i] - r["cost"]) <= 1e-12 * r["cost"]
        near = abs(r["min_clearance"]) < 1e-4 or abs(r["goal_dist"] - prob.goal_r) < 1e-4
        if not near:
            assert bool(valid[i]) == r["valid"], i
            agree += 1
    assert agree >= 12


def _planned_quad_trajectories(kpx, want=3):
    out = []
    for seed in range(12):
        prob = scenes.quad_scene(seed, clutter=120, certify=False, walls=False, tree_cap=1 << 16, lam=32)
        pl = kpx.Planner(prob)
        pl.iterate(120)
        tr = pl.best_trajectory()
        pl.close()
        if tr is not None and len(tr["steps"]) >= 2:
            out.append((prob, tr))
        if len(out) >= want:
            break
    return out


def test_refine_planner_trajectories_revalidated_fp64(kpx, rf):
    found = _planned_quad_trajectories(kpx)
    assert found, "no quadcopter problem solved"
    accepted = 0
    for prob, tr in found:
        batch = rf.Batch.from_trajectories(prob, [tr])
        valid0, cost0, _ = rf.validate(batch)
        assert bool(valid0[0])  # the planner's own trajectory, re-rolled with its own stepper
        spec = rf.default_cost(prob, w_goal=50.0)
        res = rf.refine(batch, spec, iters=30, lr=0.01)
        n = len(tr["steps"])
        u_new = res["u"][0, :n].cpu().numpy()
        J0, J = res["J0"][0].item(), res["J"][0].item()
        r = oracle.validate_controls(prob, np.asarray(tr["states"][0], np.float64), u_new, tr["steps"])
        assert r["valid"], r  # the FP64 oracle confirms the returned controls
        assert abs(res["cost"][0].item() - r["cost"]) <= 1e-12 * r["cost"]
        if bool(res["accepted"][0]):
            accepted += 1
            assert J < J0
            J64 = oracle.refine_cost(prob, spec, np.asarray(tr["states"][0], np.float64), u_new.astype(np.float64),
                                     tr["steps"])
            assert abs(J64 - J) <= 1e-3 * abs(J64)
        print("refinement: J %.5f -> %.5f, effort+duration cost %.5f -> %.5f, accepted %s"
              % (J0, J, res["cost0"][0].item(), res["cost"][0].item(), bool(res["accepted"][0])))
    assert accepted >= 1


def test_box_grid_equals_every_box(rf):
    """The box grid keeps exactly the terms of the every-box sum: the
    objective with the grid (evaluate) against the same call without a
    workspace (every box at every step), up to FP32 summation order; its
    candidates are a small part of the boxes, and every term found by
    brute force is among them."""
    import ctypes as C
    prob, x0, u, steps, n_seg, obs = _case(8, (6, 30), (10, 50), 300, seed=7)
    batch = rf.Batch(prob, x0, u, steps, n_seg, obstacles=obs)
    J_grid = rf.evaluate(batch, SPEC).cpu().numpy()
    f_cand, f_near, _, _ = rf.box_tests(batch)
    L = rf._lib()
    J_all = torch.empty(batch.count, dtype=torch.float32, device="cuda")
    cost = rf._cost_struct(SPEC)
    s = torch.cuda.current_stream()
    rf._check(L.kpx_refine_eval(C.byref(batch.dyn), C.byref(cost), C.c_void_p(batch.obs.data_ptr()),
                                int(batch.obs.shape[0]), batch.count, batch.max_segments,
                                C.c_void_p(batch.x0.data_ptr()), C.c_void_p(batch.u.data_ptr()),
                                C.c_void_p(batch.steps.data_ptr()), C.c_void_p(batch.n_seg.data_ptr()),
                                C.c_void_p(batch.order.data_ptr()), batch.max_total_steps,
                                C.c_void_p(J_all.data_ptr()), None, None, C.c_size_t(0), C.c_void_p(s.cuda_stream)),
              "kpx_refine_eval")
    J_all = J_all.cpu().numpy()
    assert np.all(np.abs(J_grid - J_all) <= 1e-5 * np.abs(J_all)), (J_grid, J_all)
    every = int(np.asarray(steps).sum()) * len(obs)
    print("box grid: %d candidates, %d terms, of %d box tests without it" % (f_cand, f_near, every))
    assert 0 < f_near <= f_cand < every // 4
    # a gradient call counts its forward and backward box tests; the same grid and points
    _, g = rf.evaluate(batch, SPEC, grad=True)
    c = rf.box_tests(batch)
    assert c[0] == f_cand and c[1] == f_near and c[2] == f_cand and c[3] == f_near
