"""Serving engine: continuous batching of trajectory checks against the latest
cloud.  Every served result is checked against the FP64 oracle (distance within
1e-5 m, arg-min attaining the oracle minimum within it; the surrogate form against
the surrogate's own oracle where the network decided), and must also be the same
alone (check_trajectory on the same cloud) and in the mix, bit for bit; admission
respects the memory budget; requests use the cloud that was current when their
batch formed.  The robots use the oracle's grids, so the oracle is the exact
reference of the served path."""
import numpy as np
import pytest

import oracle
import oracle.mlp as mlp
import scenegen as sg
from tests._gpu import DIST_TOL, assert_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


class Arm:
    def __init__(self, sc, vals, metas, robot):
        self.sc, self.vals, self.metas, self.robot = sc, vals, metas, robot

    def parity(self, q, pts, d, l, p):
        assert_parity(self.sc.dh, self.sc.base, self.vals, self.metas, q, pts, d, l, p)


@pytest.fixture(scope="module")
def world(sdf):
    ctx = sdf.Context(0, torch.cuda.current_stream())
    arms = []
    for dof, seed in ((6, 31), (7, 32)):
        sc = sg.make_scene("tiny", dof=dof, seed=seed, resolution=24)
        vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
        g = sdf.sdf_grids_upload(ctx, vals, metas)
        arms.append(Arm(sc, np.asarray(vals), [np.asarray(m) for m in metas], sdf.Robot(ctx, sc.dh, g, sc.base)))
    return ctx, arms


def _alone(sdf, ctx, robot, q, pts):
    W, N = q.shape[0], pts.shape[0]
    out = tuple(torch.empty(W, dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.int32))
    sdf.check_trajectory(ctx, robot, torch.tensor(q, dtype=torch.float32, device="cuda"), W,
                         torch.tensor(pts, dtype=torch.float32, device="cuda"), N, *out)
    assert ctx.synchronize() == 0
    return tuple(t.cpu().numpy() for t in out)


def test_results_alone_equal_in_the_mix(sdf, world):
    ctx, arms = world
    rng = np.random.default_rng(41)
    pts = sg.cloud_uniform(rng, 3000).astype(np.float32)
    # a 20 ms batch window: batches fill to max_batch (the last one waits out the window)
    srv = sdf.Server(0, slots=3, max_batch=8, max_waypoints=4096, max_points=5000, max_dof=7,
                     batch_window_us=20000)
    assert srv.set_cloud(pts) == sdf.SDF_OK
    jobs = []
    for i in range(60):
        arm = arms[i % 2]
        q = sg.spline_trajectory(rng, arm.sc.dh, 3, int(rng.integers(1, 400))).astype(np.float32)
        jobs.append((arm, q, srv.submit(arm.robot, q)))
    for arm, q, t in jobs:
        rc, d, l, p, lat = srv.poll(t, wait_us=-1)
        assert rc == sdf.SDF_OK and lat > 0
        arm.parity(q, pts, d, l, p)
        d0, l0, p0 = _alone(sdf, ctx, arm.robot, q, pts)
        assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
        assert np.array_equal(l, l0) and np.array_equal(p, p0)
    st = srv.stats()
    assert st["completed"] == 60 and st["batches"] <= 60 and st["p99_us"] >= st["p50_us"] > 0
    assert st["mean_batch"] > 1.0            # requests were batched together
    srv.close()


def test_batch_window_holds_a_lone_request(sdf, world):
    ctx, arms = world
    arm = arms[0]
    sc, robot = arm.sc, arm.robot
    rng = np.random.default_rng(44)
    pts = sg.cloud_uniform(rng, 1000).astype(np.float32)
    srv = sdf.Server(0, slots=2, max_batch=4, max_waypoints=1024, max_points=2000, max_dof=7,
                     batch_window_us=5000)
    srv.set_cloud(pts)
    q = sg.spline_trajectory(rng, sc.dh, 3, 50).astype(np.float32)
    rc, d, l, p, lat = srv.poll(srv.submit(robot, q), wait_us=-1)
    assert rc == sdf.SDF_OK and lat >= 5000.0
    arm.parity(q, pts, d, l, p)
    assert np.array_equal(d.view(np.uint32), _alone(sdf, ctx, robot, q, pts)[0].view(np.uint32))
    # four requests fill max_batch and launch without waiting out the window
    qs = [sg.spline_trajectory(rng, sc.dh, 3, 50).astype(np.float32) for _ in range(4)]
    ts = [srv.submit(robot, x) for x in qs]
    res = [srv.poll(t, wait_us=-1) for t in ts]
    assert max(r[4] for r in res) < 5000.0
    for x, r in zip(qs, res):
        arm.parity(x, pts, r[1], r[2], r[3])
    with pytest.raises(sdf.SdfError):
        sdf.Server(0, batch_window_us=-1)
    srv.close()


def test_admission_by_memory_budget(sdf, world):
    ctx, arms = world
    arm = arms[0]
    sc, robot = arm.sc, arm.robot
    rng = np.random.default_rng(42)
    pts = sg.cloud_uniform(rng, 2000).astype(np.float32)
    # the budget admits the sort scratch plus roughly one 300-waypoint request at a time
    scratch = 5000 * 16 + (5000 // 32 + 2) * 32 + 64
    budget = scratch + 300 * (6 * 4 + 12) + 100
    srv = sdf.Server(0, memory_budget_bytes=budget, slots=4, max_batch=8, max_waypoints=2048, max_points=5000,
                     max_dof=7)
    srv.set_cloud(pts)
    with pytest.raises(sdf.SdfError) as e:
        srv.submit(robot, np.zeros((1000, 6), np.float32))      # alone exceeds the budget
    assert e.value.code == sdf.SDF_ERR_OOM
    qs = [sg.spline_trajectory(rng, sc.dh, 3, 300).astype(np.float32) for _ in range(6)]
    tickets = [srv.submit(robot, q) for q in qs]
    for q, t in zip(qs, tickets):
        rc, d, l, p, _ = srv.poll(t, wait_us=-1)
        assert rc == sdf.SDF_OK
        arm.parity(q, pts, d, l, p)
        d0, _, _ = _alone(sdf, ctx, robot, q, pts)
        assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
    st = srv.stats()
    assert st["peak_in_flight"] == 1 and st["rejected"] == 1 and st["batches"] == 6
    srv.close()


def test_requests_use_the_current_cloud(sdf, world):
    ctx, arms = world
    arm = arms[1]
    sc, robot = arm.sc, arm.robot
    rng = np.random.default_rng(43)
    a = sg.cloud_uniform(rng, 2500).astype(np.float32)
    b = (sg.cloud_uniform(rng, 1800) * 0.5).astype(np.float32)
    srv = sdf.Server(0, slots=2, max_batch=4, max_waypoints=2048, max_points=5000, max_dof=7)
    q = sg.spline_trajectory(rng, sc.dh, 3, 64).astype(np.float32)
    srv.set_cloud(a)
    rc, da, la, pa, _ = srv.poll(srv.submit(robot, q), wait_us=-1)
    srv.set_cloud(b)
    rc2, db, lb, pb, _ = srv.poll(srv.submit(robot, q), wait_us=-1)
    assert rc == rc2 == sdf.SDF_OK
    arm.parity(q, a, da, la, pa)
    arm.parity(q, b, db, lb, pb)
    assert np.array_equal(da.view(np.uint32), _alone(sdf, ctx, robot, q, a)[0].view(np.uint32))
    assert np.array_equal(db.view(np.uint32), _alone(sdf, ctx, robot, q, b)[0].view(np.uint32))
    srv.close()


def test_surrogate_form_results_equal_alone(sdf, world):
    ctx, arms = world
    arm = arms[0]
    sc, robot = arm.sc, arm.robot
    grids = robot.grids
    params = sg.mlp_init(51, sc.dof + 1)
    sur = sdf.Surrogate(ctx, grids, params)
    rng = np.random.default_rng(45)
    pts = sg.cloud_uniform(rng, 2000).astype(np.float32)
    margin, eps = 0.05, 0.3
    srv = sdf.Server(0, slots=2, max_batch=4, max_waypoints=4096, max_points=5000, max_dof=7)
    srv.set_surrogate(sur, margin, eps)
    srv.set_cloud(pts)
    jobs = []
    for i in range(12):
        q = sg.spline_trajectory(rng, sc.dh, 3, int(rng.integers(1, 300))).astype(np.float32)
        jobs.append((q, srv.submit(robot, q)))
    for q, t in jobs:
        rc, d, l, p, _ = srv.poll(t, wait_us=-1)
        assert rc == sdf.SDF_OK
        W = len(q)
        out = [torch.empty(W, dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.int32)]
        sdf.check_trajectory_surrogate(ctx, robot, sur, torch.tensor(q, device="cuda"), W,
                                       torch.tensor(pts, device="cuda"), len(pts), margin, eps, *out)
        assert ctx.synchronize() == 0
        assert np.array_equal(d.view(np.uint32), out[0].cpu().numpy().view(np.uint32))
        assert np.array_equal(l, out[1].cpu().numpy()) and np.array_equal(p, out[2].cpu().numpy())
        _surrogate_form_parity(arm, params, q, pts, margin, eps, d)
    srv.set_surrogate(None)
    srv.close()


SUR_TOL = 2e-3   # the network on the GPU against its FP64 oracle (bf16 rounding order)


def _surrogate_form_parity(arm, params, q, pts, margin, eps, d):
    """Each waypoint's served distance is the grid oracle's (re-checked: surrogate
    minimum below margin + eps) or the surrogate oracle's (decided by the network);
    within SUR_TOL of the threshold either is accepted."""
    sc = arm.sc
    g_ref = oracle.check(sc.dh, sc.base, arm.vals, arm.metas, q, pts)[0]
    s_ref = mlp.check(sc.dh, sc.base, params.astype(np.float64), arm.metas, q, pts, quantize=True)[0]
    d = d.astype(np.float64)
    limit = margin + eps
    is_grid = np.abs(d - g_ref) <= DIST_TOL
    is_sur = np.abs(d - s_ref) <= SUR_TOL
    assert np.all(is_grid[s_ref < limit - SUR_TOL])
    assert np.all(is_sur[s_ref > limit + SUR_TOL])
    assert np.all(is_grid | is_sur)
