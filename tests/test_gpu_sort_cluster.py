"""The width of the cloud sort's thread-block cluster (SDF_OPT_SORT_CTAS).

The sort runs as one cluster of 8 CTAs (the portable size) or 16 (a non-portable
size, where the device can place it).  The sorted order within a Morton cell
depends on the order of shared-memory atomics, but the check's result does not:
the minimum is exact and ties are broken by the packed (distance, point, link)
key.  So both widths must give bit-identical results, and both must match the
oracle.  Clouds are ragged (not a multiple of the 32-point tile or of any CTA
share) and some carry non-finite points, which the sort drops.
"""
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


@pytest.fixture()
def ctx(sdf):
    c = sdf.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


def _widths(sdf, ctx):
    w = ctx.get_option(sdf.SDF_OPT_SORT_CTAS)
    assert w in (8, 16)
    return [8, 16] if w == 16 else [8]


def test_option_values(sdf, ctx):
    widest = ctx.get_option(sdf.SDF_OPT_SORT_CTAS)
    for bad in (-1, 1, 4, 12, 32):
        with pytest.raises(sdf.SdfError):
            ctx.set_option(sdf.SDF_OPT_SORT_CTAS, bad)
    ctx.set_option(sdf.SDF_OPT_SORT_CTAS, 8)
    assert ctx.get_option(sdf.SDF_OPT_SORT_CTAS) == 8
    if widest == 16:
        ctx.set_option(sdf.SDF_OPT_SORT_CTAS, 16)
        assert ctx.get_option(sdf.SDF_OPT_SORT_CTAS) == 16
    else:
        with pytest.raises(sdf.SdfError):
            ctx.set_option(sdf.SDF_OPT_SORT_CTAS, 16)
    ctx.set_option(sdf.SDF_OPT_SORT_CTAS, 0)
    assert ctx.get_option(sdf.SDF_OPT_SORT_CTAS) == widest


@pytest.mark.parametrize("N", [1, 31, 1013, 20_011, 333_333])
def test_widths_agree_with_each_other_and_the_oracle(sdf, ctx, N):
    sc = sg.make_scene("tiny", W=23, N=N)
    pts = np.array(sc.points, dtype=np.float32)
    if N > 100:
        pts[::97] = np.nan   # dropped by the sort
        pts[5] = np.inf
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    grids = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    finite = np.all(np.isfinite(pts), axis=1)
    keep = np.flatnonzero(finite)
    results = []
    for width in _widths(sdf, ctx):
        ctx.set_option(sdf.SDF_OPT_SORT_CTAS, width)
        rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, pts)
        # non-finite points raise the status bit but leave the rest of the check valid
        assert rc in (sdf.SDF_OK, sdf.SDF_ERR_NONFINITE) and (rc == sdf.SDF_OK) == bool(finite.all())
        results.append((d, al, ap))
    ctx.set_option(sdf.SDF_OPT_SORT_CTAS, 0)
    d0, al0, ap0 = results[0]
    for d, al, ap in results[1:]:
        assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
        assert np.array_equal(al, al0) and np.array_equal(ap, ap0)
    # the oracle on the finite points, with indices mapped back to the full cloud
    ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, pts[keep].astype(np.float64))
    ref = (ref[0], ref[1], np.where(ref[2] >= 0, keep[np.maximum(ref[2], 0)], -1))
    assert np.all(finite[ap0[ap0 >= 0]])
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, pts, d0, al0, ap0, ref=ref)
