"""check_trajectory_noalloc: the check for callers that cannot allocate GPU memory
while they run -- a fixed-period control loop that must not stall on cudaMalloc,
or a process whose memory budget is fixed at start-up.  Its scratch is a
fixed-size device array inside the library, shared by every call.

The test calls it through the C ABI twice in a row, on two different workloads,
and compares each result with check_trajectory's on the same inputs (distance
within the 1e-5 m parity tolerance, arg-min link and point equal).  The second
call runs on scratch left over from the first, which is what the call must reset.
This file is collected last so that a failure here does not hide the others.
"""
import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


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
        W, N = q.shape[0], pts.shape[0]
        d = torch.full((W,), 9.0, device="cuda")
        al = torch.full((W,), -9, dtype=torch.int32, device="cuda")
        ap = torch.full((W,), -9, dtype=torch.int32, device="cuda")
        status.fill_(7)
        rc = sdf.check_trajectory_noalloc(robot, stream, q, W, pts, N, d, al, ap, status)
        assert rc == sdf.SDF_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        rd, rl, rp = _reference(sdf, ctx, robot, q, pts)
        assert np.abs(d.cpu().numpy().astype(np.float64) - rd).max() <= TOL
        assert np.array_equal(al.cpu().numpy(), rl) and np.array_equal(ap.cpu().numpy(), rp)


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
