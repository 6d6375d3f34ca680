"""Closed-form geometry used to pin the oracle (test infrastructure).

These are textbook formulas for analytic shapes and bounds, independent of the
oracle's brute-force mesh code.
"""
import math

import numpy as np


def sdf_sphere(x, c, r):
    return np.linalg.norm(np.atleast_2d(x) - np.asarray(c), axis=1) - r


def sdf_capsule(x, p0, p1, r):
    x = np.atleast_2d(x)
    p0, p1 = np.asarray(p0, float), np.asarray(p1, float)
    seg = p1 - p0
    t = np.clip((x - p0) @ seg / (seg @ seg), 0.0, 1.0)
    return np.linalg.norm(x - (p0 + t[:, None] * seg), axis=1) - r


def sdf_box(x, c, half):
    q = np.abs(np.atleast_2d(x) - np.asarray(c)) - np.asarray(half)
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
    inside = np.minimum(np.max(q, axis=1), 0.0)
    return outside + inside


def inscribed_tolerance(mesh, p0, p1, r, t0=0, t1=None):
    """Hausdorff bound between a convex capsule (segment p0-p1, radius r) and an
    inscribed polyhedron whose vertices lie on it: the polyhedron contains every
    point within delta of the segment, delta = min over faces of the face-plane
    distance of the segment end points, so |sdf_mesh - sdf_exact| <= r - delta."""
    tris = mesh.tris[t0:t1]
    a, b, c = (mesh.verts[tris[:, k]] for k in range(3))
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d0 = np.einsum("ij,ij->i", a - np.asarray(p0), n)
    d1 = np.einsum("ij,ij->i", a - np.asarray(p1), n)
    delta = min(d0.min(), d1.min())
    assert delta > 0
    return r - delta


def point_triangle_distance_projection(p, a, b, c):
    """Independent method: project onto the plane; if the projection lies inside the
    triangle the distance is the plane distance, otherwise the nearest of the three
    edge segments."""
    p, a, b, c = (np.asarray(v, float) for v in (p, a, b, c))
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    h = (p - a) @ n
    pp = p - h * n
    inside = True
    for u, v in ((a, b), (b, c), (c, a)):
        if np.cross(v - u, pp - u) @ n < 0:
            inside = False
    if inside:
        return abs(h)

    def seg(u, v):
        t = np.clip((p - u) @ (v - u) / ((v - u) @ (v - u)), 0.0, 1.0)
        return np.linalg.norm(p - (u + t * (v - u)))
    return min(seg(a, b), seg(b, c), seg(c, a))


def interp_gap_bound(h, f):
    """|trilinear(p) - d(p)| <= h sqrt(sum_a f_a (1 - f_a)) for a 1-Lipschitz d
    sampled at nodes of spacing h (Jensen on the trilinear weights); <= sqrt(3) h / 2."""
    f = np.atleast_2d(f)
    return h * np.sqrt(np.sum(f * (1.0 - f), axis=1))


def half_diagonal(h):
    return math.sqrt(3.0) * h / 2.0
