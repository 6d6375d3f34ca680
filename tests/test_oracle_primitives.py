"""Pins for the oracle's geometric primitives (CPU only).

* Point-to-triangle distance: closed forms in each Voronoi region, an independent
  projection-based method, and dense barycentric sampling (an upper bound that
  converges from above).
* Solid angle: the octant triangle subtends pi/2, a cube face 2 pi / 3 from the
  centre; orientation flips the sign; closed meshes sum to 4 pi inside and 0 outside.
* Mesh SDF: boxes match the analytic box SDF exactly; spheres and capsules match
  within the inscribed-polyhedron Hausdorff bound; two-component unions take the
  minimum over components.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from tests import _geometry as geo

TRI = (np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))


@pytest.mark.parametrize("p,expect", [
    ((0.2, 0.2, 0.7), 0.7),                              # face interior: plane distance
    ((0.25, 0.25, -0.3), 0.3),                           # below the face
    ((-1.0, -2.0, 0.5), math.sqrt(1 + 4 + 0.25)),        # vertex a region
    ((3.0, -1.0, 0.0), math.sqrt(4 + 1)),                # vertex b region
    ((-0.5, 2.0, 1.0), math.sqrt(0.25 + 1 + 1)),         # vertex c region
    ((0.5, -2.0, 1.0), math.sqrt(4 + 1)),                # edge ab region
    ((-3.0, 0.5, 0.0), 3.0),                             # edge ac region
    ((1.0, 1.0, 0.0), math.sqrt(0.5)),                   # edge bc region
    ((1.0, 1.0, 2.0), math.sqrt(0.5 + 4)),               # edge bc region, lifted
])
def test_point_triangle_closed_forms(p, expect):
    assert oracle.point_triangle_dist(p, *TRI) == pytest.approx(expect, abs=1e-14)


def test_point_triangle_vs_projection_method_and_sampling():
    rng = np.random.default_rng(0)
    for _ in range(400):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 2.0
        d = oracle.point_triangle_dist(p, a, b, c)
        assert d == pytest.approx(geo.point_triangle_distance_projection(p, a, b, c), abs=1e-12)
    # dense barycentric sampling: every sample is on the triangle, so the sampled
    # minimum is >= the exact distance and converges to it
    a, b, c = rng.normal(size=(3, 3))
    K = 400
    i, j = np.meshgrid(np.arange(K + 1), np.arange(K + 1), indexing="ij")
    keep = i + j <= K
    u, v = i[keep] / K, j[keep] / K
    samples = a + u[:, None] * (b - a) + v[:, None] * (c - a)
    diam = max(np.linalg.norm(b - a), np.linalg.norm(c - a), np.linalg.norm(c - b))
    for _ in range(30):
        p = rng.normal(size=3) * 1.5
        d = oracle.point_triangle_dist(p, a, b, c)
        s = np.min(np.linalg.norm(samples - p, axis=1))
        assert s >= d - 1e-12
        assert s <= d + diam / K


def test_point_triangle_degenerate_falls_back_to_segments():
    a, b, c = np.zeros(3), np.array([1.0, 0, 0]), np.array([2.0, 0, 0])
    assert oracle.point_triangle_dist((1.5, 1.0, 0.0), a, b, c) == pytest.approx(1.0)
    assert oracle.point_triangle_dist((3.0, 0.0, 0.0), a, b, c) == pytest.approx(1.0)


def test_solid_angle_closed_forms():
    o = np.zeros(3)
    ex, ey, ez = np.eye(3)
    # octant triangle seen from the origin covers 1/8 of the sphere
    assert oracle.solid_angle(o, ex, ey, ez) == pytest.approx(math.pi / 2, abs=1e-14)
    assert oracle.solid_angle(o, ex, ez, ey) == pytest.approx(-math.pi / 2, abs=1e-14)
    # a cube face seen from the cube centre covers 1/6 of the sphere
    c = np.array([0.5, 0.5, 0.5])
    f = [np.array(v, float) for v in ((1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1))]
    s = oracle.solid_angle(c, f[0], f[1], f[2]) + oracle.solid_angle(c, f[0], f[2], f[3])
    assert abs(s) == pytest.approx(4 * math.pi / 6, abs=1e-13)


@pytest.mark.parametrize("mesh", [
    sg.uv_sphere_mesh([0.1, -0.2, 0.3], 0.2, 24, 12),
    sg.capsule_mesh([0, 0, 0], [0.3, 0.1, 0.0], 0.07, 16, 8),
    sg.box_mesh([0.0, 0.0, 0.0], [0.1, 0.2, 0.3], 2),
])
def test_winding_number_inside_outside(mesh):
    c = mesh.verts.mean(axis=0)
    assert oracle.winding_number(mesh, c) == pytest.approx(1.0, abs=1e-12)
    assert oracle.winding_number(mesh, c + np.array([2.0, 0.0, 0.0])) == pytest.approx(0.0, abs=1e-12)


def test_box_sdf_exact():
    rng = np.random.default_rng(1)
    c, half = np.array([0.05, -0.1, 0.2]), np.array([0.1, 0.2, 0.15])
    m = sg.box_mesh(c, half, 3)
    x = c + rng.uniform(-0.5, 0.5, size=(500, 3))
    np.testing.assert_allclose(oracle.mesh_sdf(m, x), geo.sdf_box(x, c, half), atol=1e-12)


def test_sphere_sdf_within_inscribed_bound():
    rng = np.random.default_rng(2)
    c, r = np.array([0.0, 0.1, -0.1]), 0.15
    m = sg.uv_sphere_mesh(c, r, 32, 16)
    tol = geo.inscribed_tolerance(m, c, c, r)
    x = c + rng.uniform(-0.4, 0.4, size=(500, 3))
    err = np.abs(oracle.mesh_sdf(m, x) - geo.sdf_sphere(x, c, r))
    assert err.max() <= tol + 1e-12
    assert tol < 0.01 * r


def test_capsule_sdf_within_inscribed_bound():
    rng = np.random.default_rng(3)
    p0, p1, r = np.array([-0.2, 0.0, 0.05]), np.array([0.1, 0.15, -0.05]), 0.06
    m = sg.capsule_mesh(p0, p1, r, 24, 10)
    tol = geo.inscribed_tolerance(m, p0, p1, r)
    x = rng.uniform(-0.5, 0.5, size=(800, 3))
    err = np.abs(oracle.mesh_sdf(m, x) - geo.sdf_capsule(x, p0, p1, r))
    assert err.max() <= tol + 1e-12


def test_union_is_min_over_components():
    rng = np.random.default_rng(4)
    p0, p1, r = np.array([-0.25, 0.0, 0.0]), np.zeros(3), 0.05
    half = np.array([0.06, 0.06, 0.07])
    cap = sg.capsule_mesh(p0, p1, r, 24, 10)
    m = sg.merge_meshes([cap, sg.box_mesh(np.zeros(3), half, 2)])
    tol = geo.inscribed_tolerance(cap, p0, p1, r)
    x = rng.uniform(-0.4, 0.3, size=(600, 3))
    expect = np.minimum(geo.sdf_capsule(x, p0, p1, r), geo.sdf_box(x, np.zeros(3), half))
    assert np.abs(oracle.mesh_sdf(m, x) - expect).max() <= tol + 1e-12
