"""Pins for the oracle's forward kinematics and the full per-waypoint check (CPU).

FK (standard DH, Sec. III-A "parallel forward kinematics"):
* rotations are orthonormal with det +1;
* a planar arm (all twists and offsets d zero) matches the 2-D closed form
  x = sum a_j cos(sum theta), y = sum a_j sin(sum theta);
* joint equivariance: moving joint j by delta rotates every later frame about the
  z axis of frame j-1 (catches a wrong product order or joint placement);
* the z axis of a single joint frame is (sin t sin a, -cos t sin a, cos a).

Check (Sec. III-A: map points to link frames, look up, reduce with min):
* sphere links on a planar arm: the result equals |p - centre| - r for the closest
  sphere (closed-form FK for the centres), within the interpolation gap plus the
  mesh tolerance;
* the reported value is the minimum of every (link, point) value and the reported
  arg-min attains it; ties go to the smallest point, then the smallest link;
* empty inputs: N = 0 gives +inf and -1, W = 0 gives empty outputs.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from tests import _geometry as geo

I34 = np.hstack([np.eye(3), np.zeros((3, 1))])


def _rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _h(T):
    M = np.eye(4)
    M[:3, :] = T
    return M


def test_fk_rotations_orthonormal():
    rng = np.random.default_rng(10)
    dh = sg.gen_arm(rng, 7)
    q = rng.uniform(-3, 3, size=(20, 7))
    T = oracle.fk(dh, I34, q)
    R = T[..., :3]
    np.testing.assert_allclose(np.einsum("wlji,wljk->wlik", R, R), np.broadcast_to(np.eye(3), R.shape),
                               atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)


def test_fk_planar_closed_form():
    rng = np.random.default_rng(11)
    dof = 4
    a = rng.uniform(0.1, 0.4, dof)
    dh = np.zeros((dof, 6))
    dh[:, 0] = a
    dh[:, 3] = rng.uniform(-1, 1, dof)
    q = rng.uniform(-2, 2, size=(10, dof))
    T = oracle.fk(dh, I34, q)
    for w in range(10):
        th = np.cumsum(dh[:, 3] + q[w])
        x = np.cumsum(a * np.cos(th))
        y = np.cumsum(a * np.sin(th))
        np.testing.assert_allclose(T[w, 1:, 0, 3], x, atol=1e-14)
        np.testing.assert_allclose(T[w, 1:, 1, 3], y, atol=1e-14)
        np.testing.assert_allclose(T[w, 1:, 2, 3], 0.0, atol=1e-14)
        np.testing.assert_allclose(T[w, 0], I34)


def test_fk_joint_equivariance():
    rng = np.random.default_rng(12)
    dof = 6
    dh = sg.gen_arm(rng, dof)
    base = np.hstack([_rz(0.3) @ np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0.0]]),
                      np.array([[0.1], [-0.2], [0.3]])])
    q = rng.uniform(-2, 2, dof)
    T0 = oracle.fk(dh, base, q)[0]
    for j in range(dof):
        delta = rng.uniform(-1, 1)
        q1 = q.copy()
        q1[j] += delta
        T1 = oracle.fk(dh, base, q1)[0]
        P = np.linalg.inv(_h(T0[j]))          # frame j-1 is link j's parent
        Rz = np.eye(4)
        Rz[:3, :3] = _rz(delta)
        for k in range(j + 1, dof + 1):
            np.testing.assert_allclose(P @ _h(T1[k]), Rz @ P @ _h(T0[k]), atol=1e-13)
        for k in range(0, j + 1):
            np.testing.assert_allclose(T1[k], T0[k], atol=0)


def test_fk_single_joint_axis():
    rng = np.random.default_rng(13)
    for _ in range(20):
        t, al = rng.uniform(-3, 3, 2)
        dh = np.array([[rng.uniform(0, 1), al, rng.uniform(0, 1), 0.0, -4, 4]])
        T = oracle.fk(dh, I34, np.array([[t]]))[0, 1]
        np.testing.assert_allclose(T[:, 2], [math.sin(t) * math.sin(al), -math.cos(t) * math.sin(al),
                                             math.cos(al)], atol=1e-14)
        np.testing.assert_allclose(T[:, 3], [dh[0, 0] * math.cos(t), dh[0, 0] * math.sin(t), dh[0, 2]],
                                   atol=1e-14)


def _planar_sphere_robot(rng, dof=3, r=0.05, n=20):
    a = rng.uniform(0.2, 0.35, dof)
    dh = np.zeros((dof, 6))
    dh[:, 0] = a
    dh[:, 4], dh[:, 5] = -3.0, 3.0
    meshes = [sg.uv_sphere_mesh(np.zeros(3), r, 24, 12) for _ in range(dof + 1)]
    vals, metas = oracle.build_grids(meshes, n, 0.05)
    return dh, meshes, vals, metas


def test_check_sphere_links_closed_form():
    rng = np.random.default_rng(14)
    dof, r = 3, 0.05
    dh, meshes, vals, metas = _planar_sphere_robot(rng, dof, r)
    q = rng.uniform(-2, 2, size=(12, dof))
    pts = rng.uniform(-1.2, 1.2, size=(200, 3))
    dist, al, ap = oracle.check(dh, I34, vals, metas, q, pts)
    tol = geo.inscribed_tolerance(meshes[0], np.zeros(3), np.zeros(3), r)
    for w in range(q.shape[0]):
        th = np.cumsum(q[w])
        cx = np.concatenate([[0.0], np.cumsum(dh[:, 0] * np.cos(th))])
        cy = np.concatenate([[0.0], np.cumsum(dh[:, 0] * np.sin(th))])
        centres = np.stack([cx, cy, np.zeros(dof + 1)], axis=1)
        d = np.linalg.norm(pts[None, :, :] - centres[:, None, :], axis=2) - r   # L x N
        # far points use the out-of-box rule, exact only along face axes: bound by
        # the gap at the box point plus the Lipschitz slack, so compare near points
        exact = d.min()
        assert dist[w] >= exact - geo.half_diagonal(metas[0, 3]) - tol - 1e-12
        inside = np.all(np.abs(pts[None] - centres[:, None]) < r + 0.05, axis=2)
        if inside.any():
            assert dist[w] <= d[inside].min() + geo.half_diagonal(metas[0, 3]) + tol + 1e-12


def test_check_is_min_and_argmin_attains():
    sc = sg.make_scene("tiny", W=8, N=300)
    vals, metas = oracle.build_grids(sc.meshes, 16, sc.margin)
    dist, al, ap = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)
    pv = oracle.pair_values(sc.dh, sc.base, vals, metas, sc.q, sc.points)   # W x L x N
    assert np.array_equal(dist, pv.reshape(pv.shape[0], -1).min(axis=1))
    assert np.array_equal(pv[np.arange(8), al, ap], dist)


def test_check_tie_break():
    rng = np.random.default_rng(15)
    # two coincident links (zero-length joint) and duplicated points
    dh = np.array([[0.0, 0.0, 0.0, 0.0, -3, 3]])
    m = sg.uv_sphere_mesh(np.zeros(3), 0.1, 16, 8)
    vals, metas = oracle.build_grids([m, m], 12, 0.05)
    p = rng.uniform(-0.5, 0.5, size=(5, 3))
    pts = np.concatenate([p, p[::-1]])
    q = np.zeros((3, 1))
    dist, al, ap = oracle.check(dh, I34, vals, metas, q, pts)
    best = int(np.argmin(np.linalg.norm(p, axis=1)))
    assert np.all(ap == best) and np.all(al == 0)


def test_check_empty_inputs():
    sc = sg.make_scene("tiny", W=3, N=10)
    vals, metas = oracle.build_grids(sc.meshes, 8, sc.margin)
    d, l, p = oracle.check(sc.dh, sc.base, vals, metas, sc.q, np.zeros((0, 3)))
    assert np.all(np.isinf(d)) and np.all(l == -1) and np.all(p == -1)
    d, l, p = oracle.check(sc.dh, sc.base, vals, metas, np.zeros((0, 6)), sc.points)
    assert d.shape == (0,)


def test_check_ignores_nan_points():
    sc = sg.make_scene("tiny", W=3, N=20)
    vals, metas = oracle.build_grids(sc.meshes, 8, sc.margin)
    pts = sc.points.copy()
    d0, l0, p0 = oracle.check(sc.dh, sc.base, vals, metas, sc.q, pts)
    pts2 = np.concatenate([np.full((1, 3), np.nan), pts])
    d1, l1, p1 = oracle.check(sc.dh, sc.base, vals, metas, sc.q, pts2)
    assert np.array_equal(d0, d1) and np.array_equal(p0 + 1, p1) and np.array_equal(l0, l1)


def test_fk_base_frame_left_multiplies():
    rng = np.random.default_rng(16)
    dh = sg.gen_arm(rng, 6)
    q = rng.uniform(-2, 2, size=(5, 6))
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + math.sin(0.7) * K + (1 - math.cos(0.7)) * K @ K     # Rodrigues
    base = np.hstack([R, rng.normal(size=(3, 1))])
    T_id = oracle.fk(dh, I34, q)
    T_b = oracle.fk(dh, base, q)
    for w in range(5):
        for k in range(7):
            np.testing.assert_allclose(_h(T_b[w, k]), _h(base) @ _h(T_id[w, k]), atol=1e-13)


def test_check_maps_points_into_link_frames():
    """Points placed at known link-frame positions by the FORWARD closed-form pose of
    a planar arm must be looked up at those positions (catches R versus R^T and
    translation errors, which sphere links cannot see)."""
    rng = np.random.default_rng(17)
    dof = 3
    a = rng.uniform(0.2, 0.35, dof)
    dh = np.zeros((dof, 6))
    dh[:, 0] = a
    meshes = [sg.merge_meshes([sg.capsule_mesh([-0.15, 0.02, 0.01], [0, 0, 0], 0.04, 16, 6),
                               sg.box_mesh([0.0, 0.03, 0.0], [0.05, 0.03, 0.06], 1)])
              for _ in range(dof + 1)]
    vals, metas = oracle.build_grids(meshes, 20, 0.04)
    q = rng.uniform(-2, 2, size=(4, dof))
    for w in range(4):
        th = np.concatenate([[0.0], np.cumsum(q[w])])
        tx = np.concatenate([[0.0], np.cumsum(a * np.cos(th[1:]))])
        ty = np.concatenate([[0.0], np.cumsum(a * np.sin(th[1:]))])
        for link in range(dof + 1):
            o, h, n = metas[link, :3], metas[link, 3], int(metas[link, 4])
            u = o + rng.uniform(0.05, 0.95, size=(30, 3)) * (n - 1) * h   # inside the box
            R = _rz(th[link])
            p = u @ R.T + np.array([tx[link], ty[link], 0.0])                 # forward pose
            pv = oracle.pair_values(dh, I34, vals, metas, q[w:w + 1], p)[0, link]
            ex = oracle.mesh_sdf(meshes[link], u)
            f = (u - o) / h
            f = f - np.floor(f)
            assert np.all(np.abs(pv - ex) <= geo.interp_gap_bound(h, f) + 1e-12)
