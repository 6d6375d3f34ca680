"""Pins of the Robot-SDF oracle (oracle/robot_sdf.py): hand-computed voxelisations,
and the reduction to the per-point check when every voxel lies in every block."""
import numpy as np

import oracle
import scenegen as sg
from oracle import robot_sdf as rs


def test_voxel_indices_by_hand():
    o, r, dims = np.zeros(3), 0.1, (4, 3, 2)
    pts = np.array([[0.05, 0.05, 0.05], [0.35, 0.25, 0.15], [0.45, 0.0, 0.0], [-0.01, 0.1, 0.1],
                    [0.1, 0.2, 0.1], [np.nan, 0.0, 0.0], [0.0, 0.0, 0.2]])
    # (3,2,1) -> 3 + 4 (2 + 3 1) = 23; (1,2,1) -> 1 + 4 (2 + 3) = 21
    assert list(rs.voxel_of(pts, o, r, dims)) == [0, 23, -1, -1, 21, -1, -1]
    assert list(rs.occupied(pts, o, r, dims)) == [0, 21, 23]
    lin = np.arange(24)
    assert np.array_equal(rs.voxel_of(rs.voxel_centres(lin, o, r, dims), o, r, dims), lin)
    assert np.allclose(rs.voxel_centres([23], o, r, dims), [[0.35, 0.25, 0.15]])


def test_reduces_to_the_per_point_check_at_voxel_centres():
    sc = sg.make_scene("tiny", resolution=16, W=6, N=400)
    vals, metas = oracle.build_grids(sc.meshes, 16, sc.margin)
    o, r, dims = np.array([-1.0, -1.0, -1.0]), 0.08, (25, 25, 25)
    d, v = rs.check(sc.dh, sc.base, vals, metas, sc.q, sc.points, o, r, dims, reach=100.0)
    occ = rs.occupied(sc.points, o, r, dims)
    centres = rs.voxel_centres(occ, o, r, dims)
    d_ref, l_ref, p_ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, centres)
    assert np.allclose(d, d_ref, rtol=0, atol=1e-12)
    assert np.array_equal(v, occ[p_ref])


def test_blocks_only_raise_values_and_match_inside():
    sc = sg.make_scene("tiny", resolution=16, W=4, N=400)
    vals, metas = oracle.build_grids(sc.meshes, 16, sc.margin)
    o, r, dims = np.array([-1.0, -1.0, -1.0]), 0.08, (25, 25, 25)
    occ = rs.occupied(sc.points, o, r, dims)
    full = rs.robot_sdf_values(sc.dh, sc.base, vals, metas, sc.q, occ, o, r, dims, reach=100.0)
    near = rs.robot_sdf_values(sc.dh, sc.base, vals, metas, sc.q, occ, o, r, dims, reach=0.1)
    assert np.all(near >= full - 1e-12)
    assert np.any(np.isinf(near)) and np.any(np.isfinite(near))
    # a value below the reach comes from a link whose block holds the voxel: unchanged
    small = full < 0.1
    assert np.allclose(near[small], full[small], rtol=0, atol=1e-12)


def test_voxel_gap_to_the_per_point_check_is_bounded():
    """Moving a point to its voxel centre moves it at most sqrt(3) r/2, and the
    interpolated link SDF is 1-Lipschitz per axis, so the two minima differ by at
    most sqrt(3) (sqrt(3) r / 2) (the per-axis bound summed over the axes)."""
    sc = sg.make_scene("tiny", resolution=16, W=5, N=500)
    vals, metas = oracle.build_grids(sc.meshes, 16, sc.margin)
    o, r, dims = np.array([-1.0, -1.0, -1.0]), 0.04, (50, 50, 50)
    d, _ = rs.check(sc.dh, sc.base, vals, metas, sc.q, sc.points, o, r, dims, reach=100.0)
    d_pt, _, _ = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)
    assert np.all(np.abs(d - d_pt) <= np.sqrt(3) * np.sqrt(3) * r / 2 + 1e-9)
