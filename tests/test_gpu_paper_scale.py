"""Parity at the full benchmark size (500 waypoints x 20,000 points, 7 links,
96^3 grids), in the launch configuration bench.py times.  The oracle grids are the
brute-force FP64 build (cached on disk between runs)."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from tests._gpu import assert_parity, device_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


@pytest.fixture(scope="module")
def paper():
    sc = sg.make_scene("paper")
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)
    return sc, vals, metas, ref


@pytest.fixture()
def ctx(sdf):
    c = sdf.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


def test_paper_scale_check_with_oracle_grids(sdf, ctx, paper):
    sc, vals, metas, ref = paper
    grids = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == 0
    err = assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap, ref=ref)
    print(f"paper scale max |dist - oracle| = {err:.3g} m")


def test_paper_scale_grid_build(sdf, ctx, paper):
    sc, vals, metas, _ = paper
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    gv, gm = grids.download()
    worst = max(np.abs(gv[l].astype(np.float64) - vals[l]).max() for l in range(sc.n_links))
    assert worst <= 2e-6, worst


def test_paper_scale_gpu_pipeline(sdf, ctx, paper):
    sc, vals, metas, ref = paper
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == 0
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap, ref=ref)


def test_paper_scale_point_order_invariance(sdf, ctx, paper):
    """Shuffling the cloud changes only which index names a point."""
    sc, vals, metas, ref = paper
    grids = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    perm = np.random.default_rng(0).permutation(sc.points.shape[0])
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points[perm])
    assert rc == 0
    rc0, d0, al0, ap0 = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points[perm], d, al, ap)
