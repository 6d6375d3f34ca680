"""check_trajectory_noalloc: the check for callers that cannot allocate GPU memory
while they run -- a fixed-period control loop that must not stall on cudaMalloc,
or a process whose memory budget is fixed at start-up.  Its scratch is a
fixed-size device array inside the library, shared by every call.

The tests call it through the C ABI twice in a row and compare each result with
check_trajectory's on the same inputs (distance within the 1e-5 m parity
tolerance, arg-min link and point equal) and, on a scene built from the oracle's
grids, with the FP64 oracle itself.  The second call runs on scratch left over
from the first, which is what the call must reset.  They also cover the empty
cloud and the empty trajectory, and check that a call makes no library
allocation: with the library's allocation-failure countdown armed, the call still
succeeds and the countdown is untouched.  This file is collected last so that a
failure here does not hide the others.
"""
import numpy as np
import pytest

import oracle
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


def _reference(sdf, ctx, robot, q, pts):
    W, N = q.shape[0], pts.shape[0]
    d = torch.empty(W, device="cuda")
    al = torch.empty(W, dtype=torch.int32, device="cuda")
    ap = torch.empty(W, dtype=torch.int32, device="cuda")
    sdf.check_trajectory(ctx, robot, q, W, pts, N, d, al, ap)
    assert ctx.synchronize() == sdf.SDF_OK
    return d.cpu().numpy(), al.cpu().numpy(), ap.cpu().numpy()


def _noalloc(sdf, robot, stream, q, pts, status):
    W, N = q.shape[0], pts.shape[0]
    d = torch.full((W,), 9.0, device="cuda")
    al = torch.full((W,), -9, dtype=torch.int32, device="cuda")
    ap = torch.full((W,), -9, dtype=torch.int32, device="cuda")
    status.fill_(7)
    rc = sdf.check_trajectory_noalloc(robot, stream, q, W, pts, N, d, al, ap, status)
    assert rc == sdf.SDF_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return d.cpu().numpy(), al.cpu().numpy(), ap.cpu().numpy()


def test_noalloc_matches_check_trajectory_on_two_calls(sdf):
    stream = torch.cuda.current_stream()
    ctx = sdf.Context(0, stream)
    sc = sg.make_scene("paper")
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    rng = np.random.default_rng(5)
    workloads = [
        (sc.q, sc.points),                                                      # 500 x 20,000
        (sc.q[::3] + 0.05, sc.points[rng.permutation(len(sc.points))[:7777]] + 0.01),  # 167 x 7,777
    ]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for q_np, p_np in workloads:
        q = torch.tensor(q_np, dtype=torch.float32, device="cuda")
        pts = torch.tensor(p_np, dtype=torch.float32, device="cuda")
        d, al, ap = _noalloc(sdf, robot, stream, q, pts, status)
        rd, rl, rp = _reference(sdf, ctx, robot, q, pts)
        assert np.abs(d.astype(np.float64) - rd).max() <= DIST_TOL
        assert np.array_equal(al, rl) and np.array_equal(ap, rp)


def test_noalloc_matches_the_oracle_on_two_calls(sdf):
    """Oracle grids uploaded: the allocation-free check against the FP64 oracle, a
    large cloud then a small one (the second call sees the first's leftovers)."""
    stream = torch.cuda.current_stream()
    ctx = sdf.Context(0, stream)
    sc = sg.make_scene("tiny", W=40, N=3000)
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, sdf.sdf_grids_upload(ctx, vals, metas), sc.base)
    rng = np.random.default_rng(6)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for q_np, p_np in ((sc.q, sc.points), (sc.q[::2] - 0.03, sc.points[rng.permutation(3000)[:333]] * 0.7)):
        q = torch.tensor(q_np, dtype=torch.float32, device="cuda")
        pts = torch.tensor(p_np, dtype=torch.float32, device="cuda")
        d, al, ap = _noalloc(sdf, robot, stream, q, pts, status)
        assert_parity(sc.dh, sc.base, vals, metas, q_np.astype(np.float32), p_np.astype(np.float32), d, al, ap)
        rd, rl, rp = _reference(sdf, ctx, robot, q, pts)
        assert np.abs(d.astype(np.float64) - rd).max() <= DIST_TOL
        assert np.array_equal(al, rl) and np.array_equal(ap, rp)


def test_noalloc_empty_cloud_and_empty_trajectory(sdf):
    stream = torch.cuda.current_stream()
    ctx = sdf.Context(0, stream)
    sc = sg.make_scene("tiny", W=9, N=50)
    grids = sdf.sdf_build_grids(ctx, sc.meshes, 12, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    q = torch.tensor(sc.q, dtype=torch.float32, device="cuda")
    empty = torch.zeros((0, 3), device="cuda")
    # a non-empty call first, so that the empty one runs on leftover scratch
    _noalloc(sdf, robot, stream, q, torch.tensor(sc.points, dtype=torch.float32, device="cuda"), status)
    d, al, ap = _noalloc(sdf, robot, stream, q, empty, status)
    assert np.all(np.isinf(d)) and np.all(d > 0) and np.all(al == -1) and np.all(ap == -1)
    rd, rl, rp = _reference(sdf, ctx, robot, q, empty)
    assert np.array_equal(d.view(np.uint32), rd.view(np.uint32))
    out = torch.full((1,), 3.0, device="cuda")
    idx = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    assert sdf.check_trajectory_noalloc(robot, stream, q, 0, empty, 0, out, idx, idx) == sdf.SDF_OK
    torch.cuda.synchronize()
    assert float(out.item()) == 3.0 and int(idx.item()) == 3   # W = 0 writes nothing


def test_noalloc_makes_no_library_allocation(sdf):
    stream = torch.cuda.current_stream()
    ctx = sdf.Context(0, stream)
    sc = sg.make_scene("tiny", W=20, N=500)
    grids = sdf.sdf_build_grids(ctx, sc.meshes, 12, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    q = torch.tensor(sc.q, dtype=torch.float32, device="cuda")
    pts = torch.tensor(sc.points, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = _noalloc(sdf, robot, stream, q, pts, status)      # first call on the device: set-up
    live = sdf.sdf_debug_alloc_live()[:2]
    sdf.sdf_debug_fail_alloc(1)                               # the next library allocation would fail
    try:
        for _ in range(2):
            d, al, ap = _noalloc(sdf, robot, stream, q, pts, status)
            assert np.array_equal(d.view(np.uint32), ref[0].view(np.uint32))
            assert np.array_equal(al, ref[1]) and np.array_equal(ap, ref[2])
        assert sdf.sdf_debug_alloc_live() == (*live, 1)
    finally:
        sdf.sdf_debug_fail_alloc(0)


def test_noalloc_rejects_sizes_beyond_its_scratch(sdf):
    stream = torch.cuda.current_stream()
    ctx = sdf.Context(0, stream)
    sc = sg.make_scene("tiny", W=4, N=10)
    grids = sdf.sdf_build_grids(ctx, sc.meshes, 8, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    big = sdf.SDF_NOALLOC_MAX_POINTS + 1
    pts = torch.zeros((big, 3), device="cuda")
    q = torch.zeros((4, 6), device="cuda")
    d = torch.empty(4, device="cuda")
    i = torch.empty(4, dtype=torch.int32, device="cuda")
    assert sdf.check_trajectory_noalloc(robot, stream, q, 4, pts, big, d, i, i) == sdf.SDF_ERR_INVALID_ARG
    assert sdf.check_trajectory_noalloc(robot, stream, q, -1, pts, 10, d, i, i) == sdf.SDF_ERR_INVALID_ARG
