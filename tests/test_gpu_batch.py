"""Batched uneven checks in one launch (check_batch): each request's result must
equal the same request checked alone, bit for bit, and match the oracle.

Requests differ in robot (6- and 7-DoF arms with their own grids), trajectory
length and cloud size; empty trajectories and empty clouds are mixed in."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from tests._gpu import assert_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


@pytest.fixture(scope="module")
def arms():
    """Two arm models (6- and 7-DoF) with oracle grids at a small resolution."""
    out = []
    for dof, seed in ((6, 11), (7, 12)):
        sc = sg.make_scene("tiny", dof=dof, seed=seed, resolution=20, W=4, N=10)
        vals, metas = oracle.build_grids(sc.meshes, sc.resolution, sc.margin)
        out.append((sc, vals, metas))
    return out


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda").contiguous()


def _request(rng, arm_idx, arms, W, N):
    sc, vals, metas = arms[arm_idx]
    q = sg.spline_trajectory(rng, sc.dh, 3, W) if W > 0 else np.zeros((0, sc.dof))
    pts = sg.cloud_uniform(rng, N, side=2.0)
    return arm_idx, q, pts


def test_batch_equals_standalone_and_oracle(sdf, arms):
    ctx = sdf.Context(0, torch.cuda.current_stream())
    robots = []
    for sc, vals, metas in arms:
        g = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
        robots.append(sdf.Robot(ctx, sc.dh, g, sc.base))
    rng = np.random.default_rng(21)
    shapes = [(0, 37, 1013), (1, 5, 20000), (0, 0, 50), (1, 64, 0), (0, 1, 1), (1, 200, 3333), (0, 17, 31)]
    reqs = [_request(rng, a, arms, W, N) for a, W, N in shapes]
    outs, dev_reqs = [], []
    for a, q, pts in reqs:
        W, N = q.shape[0], pts.shape[0]
        o = (torch.full((max(W, 1),), 5.0, device="cuda"), torch.full((max(W, 1),), -5, dtype=torch.int32, device="cuda"),
             torch.full((max(W, 1),), -5, dtype=torch.int32, device="cuda"))
        qd, pd = _dev(q), _dev(pts.reshape(N, 3))
        outs.append(o)
        dev_reqs.append((robots[a], qd, W, pd, N, *o))
    sdf.check_batch(ctx, dev_reqs)
    assert ctx.synchronize() == 0
    for (a, q, pts), (robot, qd, W, pd, N, *_), o in zip(reqs, dev_reqs, outs):
        if W == 0:
            continue
        d1, l1, p1 = (t[:W].cpu().numpy() for t in o)
        alone = (torch.empty(W, device="cuda"), torch.empty(W, dtype=torch.int32, device="cuda"),
                 torch.empty(W, dtype=torch.int32, device="cuda"))
        sdf.check_trajectory(ctx, robot, qd, W, pd, N, *alone)
        assert ctx.synchronize() == 0
        d0, l0, p0 = (t.cpu().numpy() for t in alone)
        assert np.array_equal(d0.view(np.uint32), d1.view(np.uint32))
        assert np.array_equal(l0, l1) and np.array_equal(p0, p1)
        sc, vals, metas = arms[a]
        assert_parity(sc.dh, sc.base, vals, metas, q, pts, d1, l1, p1)


def test_batch_of_128_small_requests_after_reserve(sdf, arms):
    ctx = sdf.Context(0, torch.cuda.current_stream())
    robots = []
    for sc, vals, metas in arms:
        g = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
        robots.append(sdf.Robot(ctx, sc.dh, g, sc.base))
    rng = np.random.default_rng(22)
    n = sdf.SDF_MAX_BATCH
    reqs = [_request(rng, i % 2, arms, int(rng.integers(1, 9)), int(rng.integers(1, 200))) for i in range(n)]
    tot_pts = sum(p.shape[0] for _, _, p in reqs)
    tot_w = sum(q.shape[0] for _, q, _ in reqs)
    tot_pairs = sum(q.shape[0] * (arms[a][0].dof + 1) for a, q, _ in reqs)
    sdf.sdf_ctx_reserve(ctx, tot_pts, tot_w, tot_pairs, n)
    dev_reqs, outs = [], []
    for a, q, pts in reqs:
        W, N = q.shape[0], pts.shape[0]
        o = (torch.empty(W, device="cuda"), torch.empty(W, dtype=torch.int32, device="cuda"),
             torch.empty(W, dtype=torch.int32, device="cuda"))
        outs.append(o)
        dev_reqs.append((robots[a], _dev(q), W, _dev(pts), N, *o))
    sdf.check_batch(ctx, dev_reqs)
    assert ctx.synchronize() == 0
    for (a, q, pts), o in zip(reqs[::9], outs[::9]):
        sc, vals, metas = arms[a]
        assert_parity(sc.dh, sc.base, vals, metas, q, pts, *(t.cpu().numpy() for t in o))
    with pytest.raises(sdf.SdfError):
        sdf.check_batch(ctx, dev_reqs + dev_reqs[:1])     # more than SDF_MAX_BATCH


def test_batch_rejects_bad_request_by_index(sdf, arms):
    ctx = sdf.Context(0, torch.cuda.current_stream())
    sc, vals, metas = arms[0]
    robot = sdf.Robot(ctx, sc.dh, sdf.sdf_grids_upload(ctx, np.stack(vals), metas), sc.base)
    q = _dev(np.zeros((3, 6)))
    d = torch.empty(3, device="cuda")
    i = torch.empty(3, dtype=torch.int32, device="cuda")
    with pytest.raises(sdf.SdfError, match="request 1"):
        sdf.check_batch(ctx, [(robot, q, 3, q, 2, d, i, i), (robot, q, 3, 0, 5, d, i, i)])
