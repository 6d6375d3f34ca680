"""The paper's Robot-SDF form of the check (Sec. III-A) on the GPU against its FP64
oracle (oracle/robot_sdf.py), and against the per-point form within the voxel gap."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from oracle import robot_sdf as rs
from tests._gpu import DIST_TOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ORIGIN, VOXEL, DIMS = np.array([-1.2, -1.2, -1.2]), 0.05, (48, 48, 48)


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


@pytest.fixture(scope="module")
def env(sdf):
    sc = sg.make_scene("tiny", W=12, N=1000)
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    ctx = sdf.Context(0, torch.cuda.current_stream())
    grids = sdf.sdf_grids_upload(ctx, vals, metas)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    return sc, ctx, robot, np.asarray(vals), [np.asarray(m) for m in metas]


def _run(sdf, ctx, robot, q, pts, reach, origin=ORIGIN, voxel=VOXEL, dims=DIMS):
    W, N = len(q), len(pts)
    d = torch.full((W,), 7.0, dtype=torch.float32, device="cuda")
    v = torch.full((W,), -7, dtype=torch.int32, device="cuda")
    pd = torch.tensor(np.asarray(pts, np.float32).reshape(-1, 3), device="cuda")
    sdf.check_trajectory_robot_sdf(ctx, robot, origin, voxel, dims, reach, torch.tensor(q, dtype=torch.float32,
                                   device="cuda"), W, pd, N, d, v)
    assert ctx.synchronize() == 0
    return d.cpu().numpy(), v.cpu().numpy()


def test_matches_oracle_within_reach(sdf, env):
    sc, ctx, robot, vals, metas = env
    reach = 0.3
    d, v = _run(sdf, ctx, robot, sc.q, sc.points, reach)
    d_ref, v_ref = rs.check(sc.dh, sc.base, vals, metas, sc.q, sc.points, ORIGIN, VOXEL, DIMS, reach)
    inner = d_ref < reach - 0.02        # away from the blocks' boundary (decided in FP32 vs FP64)
    assert inner.sum() >= 3
    assert np.max(np.abs(d[inner] - d_ref[inner])) <= DIST_TOL
    # the reported voxel attains the minimum
    for w in np.nonzero(inner)[0]:
        val = rs.robot_sdf_values(sc.dh, sc.base, vals, metas, sc.q[w:w + 1], np.array([v[w]]), ORIGIN, VOXEL,
                                  DIMS, reach)[0, 0]
        assert abs(val - d_ref[w]) <= DIST_TOL
    assert np.all(rs.voxel_of(rs.voxel_centres(v[inner], ORIGIN, VOXEL, DIMS), ORIGIN, VOXEL, DIMS) == v[inner])


def test_full_reach_is_the_per_point_check_at_voxel_centres(sdf, env):
    sc, ctx, robot, vals, metas = env
    d, v = _run(sdf, ctx, robot, sc.q, sc.points, 10.0)
    occ = rs.occupied(sc.points, ORIGIN, VOXEL, DIMS)
    d_ref, _, p_ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, rs.voxel_centres(occ, ORIGIN, VOXEL, DIMS))
    assert np.max(np.abs(d - d_ref)) <= DIST_TOL
    # within the voxel gap of the per-point form
    out = [torch.empty(len(sc.q), dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.int32)]
    sdf.check_trajectory(ctx, robot, torch.tensor(sc.q, dtype=torch.float32, device="cuda"), len(sc.q),
                         torch.tensor(sc.points, dtype=torch.float32, device="cuda"), len(sc.points), *out)
    assert ctx.synchronize() == 0
    d_pt = out[0].cpu().numpy()
    assert np.all(np.abs(d - d_pt) <= np.sqrt(3) * np.sqrt(3) * VOXEL / 2 + 1e-5)


def test_empty_and_outside(sdf, env):
    sc, ctx, robot, vals, metas = env
    d, v = _run(sdf, ctx, robot, sc.q[:3], np.zeros((0, 3)), 0.3)
    assert np.all(np.isinf(d)) and np.all(v == -1)
    d, v = _run(sdf, ctx, robot, sc.q[:3], sc.points + 10.0, 0.3)   # every point outside the grid
    assert np.all(np.isinf(d)) and np.all(v == -1)
    with pytest.raises(sdf.SdfError):
        _run(sdf, ctx, robot, sc.q[:3], sc.points, 0.3, voxel=0.0)
    with pytest.raises(sdf.SdfError):
        _run(sdf, ctx, robot, sc.q[:3], sc.points, 0.3, dims=(0, 4, 4))
