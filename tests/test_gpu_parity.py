"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-5 m per waypoint on the distance (FP32 transforms and interpolation
against FP64); the arg-min (link, point) must attain the oracle minimum to within
the same tolerance.  Cull on/off results must be bit-identical (the cull is exact).
"""
import numpy as np
import pytest

import oracle
import scenegen as sg
from tests._gpu import DIST_TOL, assert_parity, device_check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


@pytest.fixture()
def ctx(sdf):
    c = sdf.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny():
    sc = sg.make_scene("tiny", W=37, N=1013)
    vals, metas = oracle.build_grids(sc.meshes, sc.resolution, sc.margin)
    ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)
    return sc, vals, metas, ref


def _robot(sdf, ctx, sc, vals, metas):
    grids = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
    return sdf.Robot(ctx, sc.dh, grids, sc.base)


def test_grid_build_matches_oracle(sdf, ctx, tiny):
    sc, vals, metas, _ = tiny
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    gv, gm = grids.download()
    for l in range(sc.n_links):
        np.testing.assert_allclose(gm[l]["origin"], metas[l, :3], atol=1e-6)
        assert gm[l]["h"] == pytest.approx(metas[l, 3], rel=1e-6)
        assert gm[l]["radius"] >= metas[l, 8]
        err = np.abs(gv[l].astype(np.float64) - vals[l])
        assert err.max() <= 2e-6, (l, err.max())


def test_fk_matches_oracle(sdf, ctx):
    rng = np.random.default_rng(3)
    for dof in (1, 6, 7, 15):
        dh = sg.gen_arm(rng, dof)
        metas = np.zeros((dof + 1, 10))
        metas[:, 3], metas[:, 4] = 0.01, 4
        metas[:, 5:8] = rng.normal(size=(dof + 1, 3)) * 0.1
        metas[:, 8] = 0.2
        grids = sdf.sdf_grids_upload(ctx, np.zeros((dof + 1, 64)), metas)
        base = np.hstack([np.linalg.qr(rng.normal(size=(3, 3)))[0] * np.sign(1.0), rng.normal(size=(3, 1))])
        if np.linalg.det(base[:, :3]) < 0:
            base[:, 0] *= -1
        robot = sdf.Robot(ctx, dh, grids, base)
        W = 33
        q = rng.uniform(-3, 3, size=(W, dof))
        qd = torch.tensor(q, dtype=torch.float32, device="cuda")
        out = torch.empty((W, dof + 1, 16), dtype=torch.float32, device="cuda")
        sdf.sdf_forward_kinematics(ctx, robot, qd, W, out)
        assert ctx.synchronize() == 0
        o = out.cpu().numpy().astype(np.float64)
        # reference from FP32-rounded inputs so only the kinematics is compared
        T = oracle.fk(dh.astype(np.float32).astype(np.float64), base.astype(np.float32).astype(np.float64),
                      q.astype(np.float32).astype(np.float64))
        R, t = T[..., :3], T[..., 3]
        Rt = np.swapaxes(R, -1, -2)
        np.testing.assert_allclose(o[..., :12].reshape(W, dof + 1, 3, 4)[..., :3], Rt, atol=2e-6)
        np.testing.assert_allclose(o[..., :12].reshape(W, dof + 1, 3, 4)[..., 3],
                                   -np.einsum("wlij,wlj->wli", Rt, t), atol=5e-6)
        c = np.einsum("wlij,lj->wli", R, metas[:, 5:8].astype(np.float32)) + t
        np.testing.assert_allclose(o[..., 12:15], c, atol=5e-6)


@pytest.mark.parametrize("tb", [1, 2, 4])
@pytest.mark.parametrize("warps", [8, 16])
@pytest.mark.parametrize("tw", [0, 1, 2, 3])
@pytest.mark.parametrize("cull", [1, 0])
def test_check_tiny_all_launch_shapes(sdf, ctx, tiny, tw, cull, warps, tb):
    # 16-warp blocks hold two waypoints of the 7-link arm; the 19 blocks of W = 37
    # are one wave, so they take interleaved waypoints (b and b + 19); tb tiles a
    # warp takes per step in phase B
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    ctx.set_option(sdf.SDF_OPT_BLOCK_WARPS, warps)
    ctx.set_option(sdf.SDF_OPT_WAYPOINTS_PER_BLOCK, tw)
    ctx.set_option(sdf.SDF_OPT_CULL, cull)
    ctx.set_option(sdf.SDF_OPT_TILE_BATCH, tb)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap, ref=ref)


@pytest.mark.parametrize("stride", [3, 4])
def test_cull_is_exact_bitwise(sdf, ctx, tiny, stride):
    sc, vals, metas, _ = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    ctx.set_option(sdf.SDF_OPT_POINT_STRIDE, stride)
    outs = []
    for cull in (1, 0):
        ctx.set_option(sdf.SDF_OPT_CULL, cull)
        for tw in (1, 2):
            ctx.set_option(sdf.SDF_OPT_WAYPOINTS_PER_BLOCK, tw)
            rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points, stride=stride)
            assert rc == 0
            outs.append((d.view(np.uint32).copy(), al.copy(), ap.copy()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


def test_host_buffers_match_device(sdf, ctx, tiny):
    sc, vals, metas, _ = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    W, N = sc.q.shape[0], sc.points.shape[0]
    hd = np.empty(W, np.float32)
    hl = np.empty(W, np.int32)
    hp = np.empty(W, np.int32)
    rc2 = sdf.check_trajectory_host(ctx, robot, np.ascontiguousarray(sc.q, np.float32), W,
                                    np.ascontiguousarray(sc.points, np.float32), N, hd, hl, hp)
    assert rc == rc2 == 0
    assert np.array_equal(d.view(np.uint32), hd.view(np.uint32))
    assert np.array_equal(al, hl) and np.array_equal(ap, hp)


def test_edge_cases(sdf, ctx, tiny):
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    # N = 0: +inf and -1
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, np.zeros((0, 3)))
    assert rc == 0 and np.all(np.isinf(d)) and np.all(al == -1) and np.all(ap == -1)
    # W = 0: no-op
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, np.zeros((0, 6)), sc.points)
    assert rc == 0 and d.shape == (0,)
    # W = 1 and N = 1
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q[:1], sc.points[:1])
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q[:1], sc.points[:1], d, al, ap)
    # every point far outside every grid box (out-of-box rule everywhere)
    far = sc.points * 0.1 + np.array([5.0, -4.0, 3.0])
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, far)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, far, d, al, ap)
    # points exactly on grid box faces and nodes of link 0 (base frame = world)
    o, h, n = metas[0, :3], metas[0, 3], int(metas[0, 4])
    rng = np.random.default_rng(9)
    face = o + rng.integers(0, n, size=(300, 3)) * h
    face[:100, 0] = o[0]
    face[100:200, 1] = o[1] + (n - 1) * h
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, face)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, face, d, al, ap)


def test_penetration_gives_negative_distance(sdf, ctx, tiny):
    sc, vals, metas, _ = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    T = oracle.fk(sc.dh, sc.base, sc.q)                  # points at link-sphere centres
    pts = np.einsum("wlij,lj->wli", T[..., :3], metas[:, 5:8]) + T[..., 3]
    pts = pts.reshape(-1, 3)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, pts)
    assert rc == 0 and np.all(d < 0)
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, pts, d, al, ap)


def test_nonfinite_inputs_flagged(sdf, ctx, tiny):
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    pts = np.concatenate([np.full((1, 3), np.nan), sc.points])
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, pts)
    assert rc == sdf.SDF_ERR_NONFINITE
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, pts, d, al, ap)
    assert ctx.synchronize() == 0          # status was cleared
    # an infinite joint value poisons the links after that joint only; the
    # earlier links still give finite distances (as in the oracle)
    q = sc.q.copy()
    q[3, 2] = np.inf
    q[5, 0] = np.nan          # first joint: every moving link is NaN, base link stays
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, q, sc.points)
    assert rc == sdf.SDF_ERR_NONFINITE
    assert al[3] in (0, 1, 2) and al[5] == 0
    assert_parity(sc.dh, sc.base, vals, metas, q, sc.points, d, al, ap)


def test_invalid_arguments(sdf, ctx, tiny):
    sc, vals, metas, _ = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    d = torch.empty(4, device="cuda")
    i = torch.empty(4, dtype=torch.int32, device="cuda")
    q = torch.zeros((4, 6), device="cuda")
    with pytest.raises(sdf.SdfError) as e:
        sdf.check_trajectory(ctx, robot, q, 4, 0, 10, d, i, i)
    assert e.value.code == sdf.SDF_ERR_INVALID_ARG
    with pytest.raises(sdf.SdfError):
        sdf.check_trajectory(ctx, robot, q, 4, q, sdf.SDF_MAX_POINTS + 1, d, i, i)
    with pytest.raises(sdf.SdfError):
        ctx.set_option(sdf.SDF_OPT_POINT_STRIDE, 5)
    with pytest.raises(sdf.SdfError):
        ctx.set_option(sdf.SDF_OPT_WAYPOINTS_PER_BLOCK, 17)
    with pytest.raises(sdf.SdfError):
        sdf.Robot(ctx, sc.dh[:3], robot.grids, sc.base)     # 4 links vs 7 grids


def test_deterministic_repeat(sdf, ctx, tiny):
    sc, vals, metas, _ = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    ctx.set_option(sdf.SDF_OPT_WAYPOINTS_PER_BLOCK, 1)
    a = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    b = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_gpu_pipeline_end_to_end(sdf, ctx, tiny):
    """GPU-built grids + GPU check against oracle grids + oracle check."""
    sc, vals, metas, ref = tiny
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap, ref=ref)


def test_sixteen_links(sdf, ctx):
    """A 15-DoF arm (16 links, the most a robot has): a block then holds one waypoint's
    16 (waypoint, link) pairs, every bit of the per-tile pair masks is in use, and the
    8-warp block form is not available.  Parity with the oracle, culled and unculled
    results bit-identical."""
    sc = sg.make_scene("tiny", dof=15, n_lon=8, n_lat=4, W=24, N=700)
    vals, metas = oracle.build_grids(sc.meshes, sc.resolution, sc.margin)
    ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)
    robot = _robot(sdf, ctx, sc, vals, metas)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap, ref=ref)
    ctx.set_option(sdf.SDF_OPT_CULL, 0)
    try:
        rc, d0, al0, ap0 = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    finally:
        ctx.set_option(sdf.SDF_OPT_CULL, 1)
    assert rc == 0
    assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
    assert np.array_equal(al, al0) and np.array_equal(ap, ap0)


@pytest.mark.parametrize("N,tb", [(4096 * 32 - 5, 1), (4096 * 32, 1), (4096 * 32, 4), (4096 * 32 + 1, 1),
                                  (4096 * 32 + 1, 2), (4096 * 32 + 1, 4)])
def test_staged_and_flat_phase_b_boundary(sdf, ctx, tiny, N, tb):
    """Clouds on either side of 4,096 tiles: at most that many tile spheres are staged
    in shared memory and phase B is grouped by tile; one more tile and the flat
    (pair, tile) list is used.  Both against the oracle."""
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    rng = np.random.default_rng(N)
    pts = rng.uniform(-1.2, 1.2, (N, 3))
    q = sc.q[:6]
    ctx.set_option(sdf.SDF_OPT_TILE_BATCH, tb)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, q, pts)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, q, pts, d, al, ap)


def test_maximum_cloud_size(sdf, ctx, tiny):
    """N = SDF_MAX_POINTS (2^24 - 1, the largest index the packed key holds):
    the sort's loop paths and the top of the index range, against the oracle on a
    few waypoints; the arg-min may point anywhere in the cloud."""
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    N = sdf.SDF_MAX_POINTS
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    pts = (torch.rand((N, 3), generator=gen, device="cuda") * 2.4 - 1.2).contiguous()
    # the last point sits on the robot's base, so the last index wins for most waypoints
    pts[N - 1] = torch.tensor(sc.base[:, 3], dtype=torch.float32, device="cuda")
    q = sc.q[:3]
    W = len(q)
    out = [torch.full((W,), 7.0, dtype=torch.float32, device="cuda"),
           torch.full((W,), -7, dtype=torch.int32, device="cuda"), torch.full((W,), -7, dtype=torch.int32, device="cuda")]
    sdf.check_trajectory(ctx, robot, torch.tensor(q, dtype=torch.float32, device="cuda"), W, pts, N, *out)
    assert ctx.synchronize() == 0
    d, al, ap = [t.cpu().numpy() for t in out]
    host = pts.cpu().numpy()
    del pts
    assert_parity(sc.dh, sc.base, vals, metas, q, host, d, al, ap)
    assert np.all(ap >= 0) and np.all(ap < N)


def test_host_calls_replay_with_new_contents(sdf, ctx, tiny):
    """Repeated host-buffer calls (replayed as one captured graph when the buffers are
    page-locked) read the buffers' current contents and follow option changes."""
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    W, N = len(sc.q), len(sc.points)
    q = torch.tensor(sc.q, dtype=torch.float32).pin_memory()
    p = torch.tensor(sc.points, dtype=torch.float32).pin_memory()
    outs = [torch.empty(W, dtype=dt).pin_memory() for dt in (torch.float32, torch.int32, torch.int32)]
    rng = np.random.default_rng(21)
    for it in range(4):
        if it == 2:
            ctx.set_option(sdf.SDF_OPT_CULL, 0)   # drops the captured graph
        qq = sc.q + rng.normal(0, 0.05, sc.q.shape) * (it > 0)
        pp = sc.points + rng.normal(0, 0.02, sc.points.shape) * (it > 0)
        q.copy_(torch.tensor(qq, dtype=torch.float32))
        p.copy_(torch.tensor(pp, dtype=torch.float32))
        rc = sdf.check_trajectory_host(ctx, robot, q.numpy(), W, p.numpy(), N, *[o.numpy() for o in outs])
        assert rc == 0
        rc2, d, al, ap = device_check(sdf, torch, ctx, robot, q.numpy(), p.numpy())
        assert rc2 == 0
        assert np.array_equal(outs[0].numpy().view(np.uint32), d.view(np.uint32))
        assert np.array_equal(outs[1].numpy(), al) and np.array_equal(outs[2].numpy(), ap)
    ctx.set_option(sdf.SDF_OPT_CULL, 1)


def test_prepared_host_check_reads_current_contents(sdf, ctx, tiny):
    """sdf.HostCheck binds the five page-locked buffers once; every call re-reads their
    contents, returns promptly with the results in place, and agrees bitwise with the
    device path; a non-finite point still comes back as SDF_ERR_NONFINITE."""
    sc, vals, metas, ref = tiny
    robot = _robot(sdf, ctx, sc, vals, metas)
    W, N = len(sc.q), len(sc.points)
    q = torch.tensor(sc.q, dtype=torch.float32).pin_memory()
    p = torch.tensor(sc.points, dtype=torch.float32).pin_memory()
    outs = [torch.empty(W, dtype=dt).pin_memory() for dt in (torch.float32, torch.int32, torch.int32)]
    call = sdf.HostCheck(ctx, robot, q.numpy(), W, p.numpy(), N, *[o.numpy() for o in outs])
    rng = np.random.default_rng(22)
    for it in range(6):
        qq = sc.q + rng.normal(0, 0.05, sc.q.shape) * (it > 0)
        pp = sc.points + rng.normal(0, 0.02, sc.points.shape) * (it > 0)
        q.copy_(torch.tensor(qq, dtype=torch.float32))
        p.copy_(torch.tensor(pp, dtype=torch.float32))
        outs[0].fill_(float("nan"))
        assert call() == 0
        rc2, d, al, ap = device_check(sdf, torch, ctx, robot, q.numpy(), p.numpy())
        assert rc2 == 0
        assert np.array_equal(outs[0].numpy().view(np.uint32), d.view(np.uint32))
        assert np.array_equal(outs[1].numpy(), al) and np.array_equal(outs[2].numpy(), ap)
        if it == 0:
            assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, outs[0].numpy(), outs[1].numpy(),
                          outs[2].numpy(), ref=ref)
    p[3, 1] = float("nan")
    assert call() == sdf.SDF_ERR_NONFINITE
    p[3, 1] = 0.0
    assert call() == 0
