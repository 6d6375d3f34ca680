"""The full batched workload (64 uneven checks, 6- and 7-DoF arms, 96^3 grids) in
one launch: every request equals its standalone check bit for bit, a CUDA-graph
replay equals the direct launch, and sampled waypoints match the FP64 oracle."""
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
def setup(sdf):
    bs = sg.make_batched()
    stream = torch.cuda.Stream()
    ctx = sdf.Context(0, stream)
    robots = [sdf.Robot(ctx, a.dh, sdf.sdf_build_grids(ctx, a.meshes, a.resolution, a.margin), a.base)
              for a in bs.arms]
    reqs, outs = [], []
    for a, q, p in bs.instances:
        W, N = q.shape[0], p.shape[0]
        o = tuple(torch.full((W,), -3, dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.int32))
        outs.append(o)
        reqs.append((robots[a], torch.tensor(q, dtype=torch.float32, device="cuda"), W,
                     torch.tensor(p, dtype=torch.float32, device="cuda"), N, *o))
    return bs, ctx, stream, robots, reqs, outs


def _fetch(outs):
    return [tuple(t.cpu().numpy().copy() for t in o) for o in outs]


def test_batched_equals_standalone(sdf, setup):
    bs, ctx, stream, robots, reqs, outs = setup
    sdf.check_batch(ctx, reqs)
    assert ctx.synchronize() == 0
    batch = _fetch(outs)
    for r, b in zip(reqs, batch):
        robot, q, W, p, N = r[:5]
        alone = tuple(torch.empty(W, dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.int32))
        sdf.check_trajectory(ctx, robot, q, W, p, N, *alone)
        assert ctx.synchronize() == 0
        a = tuple(t.cpu().numpy() for t in alone)
        assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_graph_replay_equals_direct(sdf, setup):
    bs, ctx, stream, robots, reqs, outs = setup
    sdf.check_batch(ctx, reqs)
    assert ctx.synchronize() == 0
    direct = _fetch(outs)
    for o in outs:
        for t in o:
            t.fill_(-9)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sdf.check_batch(ctx, reqs)
    for o in outs:
        for t in o:
            t.fill_(-9)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(direct, _fetch(outs)):
        assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_batched_sampled_oracle_parity(sdf, setup):
    bs, ctx, stream, robots, reqs, outs = setup
    sdf.check_batch(ctx, reqs)
    assert ctx.synchronize() == 0
    res = _fetch(outs)
    grids = [oracle.build_grids_cached(a.meshes, a.resolution, a.margin) for a in bs.arms]
    rng = np.random.default_rng(4)
    for i in rng.choice(len(bs.instances), 8, replace=False):
        a, q, p = bs.instances[i]
        arm = bs.arms[a]
        vals, metas = grids[a]
        ws = rng.choice(q.shape[0], 3, replace=False)
        d, l, pt = (x[ws] for x in res[i])
        assert_parity(arm.dh, arm.base, vals, metas, q[ws], p, d, l, pt)


def test_autotune_then_check(sdf, setup):
    bs, ctx, stream, robots, reqs, outs = setup
    sub = reqs[:4]
    tw, tb, us = sdf.sdf_autotune(ctx, sub, repeats=2)
    assert 1 <= tw <= 2 and tb in (1, 2, 4) and us > 0
    sdf.check_batch(ctx, sub)
    assert ctx.synchronize() == 0
