"""The hardware trilinear option (SDF_OPT_TEX3D): the grid lookup by the texture
unit's filter instead of the FP32 software interpolation.

The filter keeps each axis weight with 8 fractional bits, so a filtered value is
the exact trilinear value at a point moved by at most h/256 per axis, and the
per-axis 1-Lipschitz interpolant then differs from the FP32 one by at most
3 h / 256.  The tests measure the error against the FP64 oracle on the small and
the paper-scale scene, check it against that bound, check that culling stays
exact under the filter (culled and unculled results bit-identical), and enforce
the acceptance rule: the option is on by default only if it meets the 1e-5 m
tolerance on both scenes.
"""
import numpy as np
import pytest

import oracle
import scenegen as sg
from tests._gpu import DIST_TOL, assert_parity, device_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MEASURED = {}


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


def _setup(sdf, name):
    sc = sg.make_scene(name)
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    ctx = sdf.Context(0, torch.cuda.current_stream())
    grids = sdf.sdf_grids_upload(ctx, np.stack(vals), metas)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    return sc, np.asarray(vals), [np.asarray(m) for m in metas], ctx, grids, robot


@pytest.mark.parametrize("name", ["tiny", "paper"])
def test_tex3d_error_against_the_oracle(sdf, name):
    sc, vals, metas, ctx, grids, robot = _setup(sdf, name)
    ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)
    assert ctx.get_option(sdf.SDF_OPT_TEX3D) == 0
    ctx.set_option(sdf.SDF_OPT_TEX3D, 1)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == sdf.SDF_OK
    h = max(float(m[3]) for m in metas)
    bound = 3.0 * h / 256.0 + 1e-6
    err = np.abs(d.astype(np.float64) - ref[0]).max()
    assert err <= bound, (err, bound)
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap, ref=ref, tol=2.0 * bound)
    # the software path on the same context, for comparison
    ctx.set_option(sdf.SDF_OPT_TEX3D, 0)
    rc, d0, al0, ap0 = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == sdf.SDF_OK
    err0 = np.abs(d0.astype(np.float64) - ref[0]).max()
    assert err0 <= DIST_TOL
    MEASURED[name] = err
    print(f"{name}: h = {h * 1e3:.2f} mm, max |tex3d - oracle| = {err:.3g} m (bound {bound:.3g}), "
          f"FP32 software path {err0:.3g} m")


def test_tex3d_culling_is_exact(sdf):
    sc, vals, metas, ctx, grids, robot = _setup(sdf, "tiny")
    ctx.set_option(sdf.SDF_OPT_TEX3D, 1)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    ctx.set_option(sdf.SDF_OPT_CULL, 0)
    rc0, d0, al0, ap0 = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == rc0 == sdf.SDF_OK
    assert np.array_equal(d.view(np.uint32), d0.view(np.uint32))
    assert np.array_equal(al, al0) and np.array_equal(ap, ap0)
    # the texture copy leaves the grids as they were
    gv, _ = grids.download()
    assert np.array_equal(gv.reshape(len(metas), -1), np.stack(vals).astype(np.float32))


def test_tex3d_default_follows_the_tolerance(sdf):
    """On by default only if it met 1e-5 m on both scenes."""
    if len(MEASURED) < 2:
        pytest.skip("needs both error measurements")
    ctx = sdf.Context(0, torch.cuda.current_stream())
    meets = max(MEASURED.values()) <= DIST_TOL
    assert ctx.get_option(sdf.SDF_OPT_TEX3D) == (1 if meets else 0)
