"""Gather-roofline measurement: plausible, positive rates on resident grids."""
import math

import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_measure_gather_rates():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as sdf
    ctx = sdf.Context(0, torch.cuda.current_stream())
    sc = sg.make_scene("tiny", resolution=48)
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    g, c = sdf.sdf_measure_gather(ctx, grids)
    assert math.isfinite(g) and math.isfinite(c)
    # a cell read is 8 loads (4 pairs of neighbours): slower than one random load,
    # faster than 8 independent ones; both far above 1e9/s and below 1e14/s
    assert 1e9 < c < g < 1e14
    assert c > g / 8
    with pytest.raises(sdf.SdfError):
        sdf.sdf_measure_gather(ctx, sdf.Grids(ctx, None))
