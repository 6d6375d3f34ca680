"""Pins for the oracle's Link SDF grids and lookup (CPU only).

* Grid geometry: the box holds the mesh plus the margin, spacing is isotropic.
* Node values match analytic sphere / capsule / box SDFs within the mesh tolerance.
* 1-Lipschitz: node values never change faster than the node distance.
* Exact nodes: lookups at node positions return the stored value (pins layout,
  origin and index order).
* Interpolation gap: |lookup(p) - mesh_sdf(p)| <= h sqrt(sum f(1-f)) <= sqrt(3) h / 2
  (the per-grid half of the clearance threshold printed in Sec. IV-C).
* Out-of-box rule: continuous at the faces, exact along a sphere's axis through a
  face centre up to the gap at the face point.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenegen as sg
from tests import _geometry as geo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


@pytest.fixture(scope="module")
def sphere_grid():
    c, r = np.array([0.02, -0.01, 0.03]), 0.12
    m = sg.uv_sphere_mesh(c, r, 32, 16)
    vals, meta = oracle.build_grid(m, 24, 0.05)
    return m, c, r, vals, meta


def _nodes(meta):
    n = int(meta[4])
    i = np.arange(n)
    k, j, ii = np.meshgrid(i, i, i, indexing="ij")
    return meta[:3] + meta[3] * np.stack([ii.ravel(), j.ravel(), k.ravel()], axis=1)


def test_grid_meta_geometry():
    m = sg.capsule_mesh([-0.3, 0.05, 0.0], [0.0, 0.0, 0.0], 0.06, 16, 8)
    meta = oracle.grid_meta(m, 32, 0.05)
    lo, hi = m.verts.min(0), m.verts.max(0)
    o, h, n = meta[:3], meta[3], int(meta[4])
    top = o + (n - 1) * h
    assert np.all(o <= lo - 0.05 + 1e-12) and np.all(top >= hi + 0.05 - 1e-12)
    span = (hi - lo).max() + 0.1
    assert h == pytest.approx(span / (n - 1), rel=1e-14)
    np.testing.assert_allclose((o + top) / 2, (lo + hi) / 2, atol=1e-14)
    # bounding sphere holds every vertex, and touches one
    dv = np.linalg.norm(m.verts - meta[5:8], axis=1)
    assert dv.max() == pytest.approx(meta[8], rel=1e-14)


def test_sphere_grid_matches_analytic(sphere_grid):
    m, c, r, vals, meta = sphere_grid
    tol = geo.inscribed_tolerance(m, c, c, r)
    err = np.abs(vals - geo.sdf_sphere(_nodes(meta), c, r))
    assert err.max() <= tol + 1e-12


def test_capsule_and_box_grids_match_analytic():
    p0, p1, r = np.array([-0.2, 0.03, -0.02]), np.zeros(3), 0.05
    cap = sg.capsule_mesh(p0, p1, r, 20, 8)
    vals, meta = oracle.build_grid(cap, 20, 0.04)
    tol = geo.inscribed_tolerance(cap, p0, p1, r)
    assert np.abs(vals - geo.sdf_capsule(_nodes(meta), p0, p1, r)).max() <= tol + 1e-12
    half = np.array([0.05, 0.08, 0.03])
    box = sg.box_mesh(np.zeros(3), half, 1)
    vals, meta = oracle.build_grid(box, 17, 0.03)
    np.testing.assert_allclose(vals, geo.sdf_box(_nodes(meta), np.zeros(3), half), atol=1e-12)


def test_grid_is_one_lipschitz():
    scene = sg.make_scene("tiny")
    vals, meta = oracle.build_grid(scene.meshes[3], 20, 0.05)
    x = _nodes(meta)
    rng = np.random.default_rng(5)
    a = rng.integers(0, vals.size, 20000)
    b = rng.integers(0, vals.size, 20000)
    assert np.all(np.abs(vals[a] - vals[b]) <= np.linalg.norm(x[a] - x[b], axis=1) + 1e-12)
    n = int(meta[4])
    g = vals.reshape(n, n, n)   # [k][j][i]
    for axis in range(3):
        assert np.abs(np.diff(g, axis=axis)).max() <= meta[3] + 1e-12


def test_exact_nodes(sphere_grid):
    m, c, r, vals, meta = sphere_grid
    x = _nodes(meta)
    rng = np.random.default_rng(6)
    pick = rng.choice(vals.size, 3000, replace=False)
    # every node, including the last row / column / layer (upper-face clamp)
    n = int(meta[4])
    corner = np.array([n ** 3 - 1, n - 1, n * n - 1, (n - 1) * n * n])
    pick = np.concatenate([pick, corner])
    # node positions round in FP64, so u lands within ~1e-15 of the integer; a
    # wrong layout or index order would be off by a node-to-node step (~h)
    np.testing.assert_allclose(oracle.lookup(vals, meta, x[pick]), vals[pick], rtol=0, atol=1e-13)
    assert meta[3] > 1e-3


def test_interpolation_gap_bound():
    scene = sg.make_scene("tiny")
    mesh = scene.meshes[2]
    vals, meta = oracle.build_grid(mesh, 16, 0.05)
    o, h, n = meta[:3], meta[3], int(meta[4])
    rng = np.random.default_rng(7)
    p = o + rng.uniform(0, (n - 1) * h, size=(3000, 3))
    u = (p - o) / h
    f = u - np.minimum(np.floor(u), n - 2)
    gap = np.abs(oracle.lookup(vals, meta, p) - oracle.mesh_sdf(mesh, p))
    bound = geo.interp_gap_bound(h, f)
    assert np.all(gap <= bound + 1e-12)
    assert np.all(bound <= geo.half_diagonal(h) + 1e-15)
    # the bound is not vacuous: the gap is a visible fraction of it somewhere
    assert gap.max() > 0.05 * bound.max()


def test_half_diagonal_reproduces_paper_clearance():
    g = json.load(open(GOLDEN))["clearance_threshold"]
    total = geo.half_diagonal(g["env_voxel_m"]) + geo.half_diagonal(g["link_sdf_resolution_m"])
    assert round(total, g["printed_digits"]) == pytest.approx(g["printed_value_m"])


def test_out_of_box_rule(sphere_grid):
    m, c, r, vals, meta = sphere_grid
    o, h, n = meta[:3], meta[3], int(meta[4])
    top = o + (n - 1) * h
    tol = geo.inscribed_tolerance(m, c, c, r)
    # continuity at every face: stepping eps outward adds eps
    rng = np.random.default_rng(8)
    for axis in range(3):
        for side in (0, 1):
            q = o + rng.uniform(0, (n - 1) * h, size=(50, 3))
            q[:, axis] = top[axis] if side else o[axis]
            eps = 1e-6
            p = q.copy()
            p[:, axis] += eps if side else -eps
            np.testing.assert_allclose(oracle.lookup(vals, meta, p),
                                       oracle.lookup(vals, meta, q) + eps, atol=1e-12)
    # along the axis through a face centre the sphere distance is additive, so
    # the rule is exact up to the interpolation gap at the face point (<= sqrt3 h/2)
    mid = (o + top) / 2
    for axis in range(3):
        for dist in (0.05, 0.3, 1.0):
            p = np.array(mid, dtype=float)
            p[axis] = top[axis] + dist
            p[(axis + 1) % 3] = c[(axis + 1) % 3]
            p[(axis + 2) % 3] = c[(axis + 2) % 3]
            g = oracle.lookup(vals, meta, p)[0]
            d = geo.sdf_sphere(p, c, r)[0]
            assert abs(g - d) <= geo.half_diagonal(h) + tol + 1e-12
    # corners: distance to the box is the Euclidean distance to the corner
    p = top + np.array([0.3, 0.4, 1.2])
    g = oracle.lookup(vals, meta, p)[0]
    assert g == pytest.approx(1.3 + vals[-1], abs=1e-12)
