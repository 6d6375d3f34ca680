"""FP64 CPU oracle for the batched runtime distance check (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never loads it and shares no code with it.

The arithmetic lives in ``sdf_oracle.c`` (plain C, double precision, OpenMP over
independent outputs only); this module compiles it with gcc and marshals numpy
arrays.  Each function names the part of the paper it follows:

* ``build_grid`` / ``grid_meta`` -- Link SDFs sampled on a grid in the link frame
  (Sec. III-A).  Brute-force signed point-to-mesh distance, sign by winding number.
* ``fk`` -- parallel forward kinematics per configuration (Sec. III-A), standard DH.
* ``lookup`` -- trilinear interpolation of a link SDF (the grid-sample interpolation
  of Sec. III-A), distance-to-box plus boundary value outside the grid box.
* ``check`` -- per-configuration min over links and obstacle points with arg-min
  (Sec. III-A, runtime reduction with min for each configuration).

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants and brute force (see the test module docstrings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_sdf_oracle.so")
_lib = None

META_LEN = 10   # origin[3], h, n, centre[3], radius, margin


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sigs = {
        "oracle_set_threads": (None, [ctypes.c_int]),
        "oracle_get_threads": (ctypes.c_int, []),
        "oracle_max_links": (ctypes.c_int, []),
        "oracle_point_triangle_dist2": (f64, [P, P, P, P]),
        "oracle_solid_angle": (f64, [P, P, P, P]),
        "oracle_winding_number": (f64, [P, P, i32, P]),
        "oracle_mesh_sdf": (f64, [P, P, P, i32, P]),
        "oracle_mesh_sdf_many": (None, [P, P, P, i32, P, i64, P]),
        "oracle_grid_meta": (None, [P, i32, i32, f64, P]),
        "oracle_build_grid": (None, [P, i32, P, P, i32, i32, f64, P, P]),
        "oracle_fk": (None, [P, i32, P, P, i64, P]),
        "oracle_lookup": (f64, [P, P, P]),
        "oracle_lookup_many": (None, [P, P, P, i64, P]),
        "oracle_check": (None, [P, i32, P, P, P, P, P, i64, P, i64, P, P, P]),
        "oracle_pair_values": (None, [P, i32, P, P, P, P, P, i64, P, i64, P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _d(a, shape_last=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape_last is not None and a.shape[-1] != shape_last:
        raise ValueError(f"expected last dim {shape_last}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


# --------------------------------------------------------------- primitives

def point_triangle_dist(p, a, b, c) -> float:
    """Euclidean distance from p to triangle abc (closest-point by Voronoi region)."""
    arrs = [_d(x) for x in (p, a, b, c)]
    return float(np.sqrt(_load().oracle_point_triangle_dist2(*[_p(x) for x in arrs])))


def solid_angle(p, a, b, c) -> float:
    """Signed solid angle of triangle abc seen from p (Van Oosterom & Strackee)."""
    arrs = [_d(x) for x in (p, a, b, c)]
    return float(_load().oracle_solid_angle(*[_p(x) for x in arrs]))


def winding_number(mesh, x) -> float:
    v, t, x = _d(mesh.verts), np.ascontiguousarray(mesh.tris, np.int32), _d(x)
    return float(_load().oracle_winding_number(_p(v), _p(t), int(t.shape[0]), _p(x)))


def mesh_sdf(mesh, x) -> np.ndarray:
    """Signed distance from each row of x (M x 3) to the mesh (min over components)."""
    x = _d(np.atleast_2d(x), 3)
    v, t = _d(mesh.verts), np.ascontiguousarray(mesh.tris, np.int32)
    off = np.ascontiguousarray(mesh.comp_offsets, np.int32)
    out = np.empty(x.shape[0])
    _load().oracle_mesh_sdf_many(_p(v), _p(t), _p(off), int(off.shape[0] - 1), _p(x),
                                 int(x.shape[0]), _p(out))
    return out


# ------------------------------------------------------------------- grids

def grid_meta(mesh, n: int, margin: float) -> np.ndarray:
    v = _d(mesh.verts)
    meta = np.empty(META_LEN)
    _load().oracle_grid_meta(_p(v), int(v.shape[0]), int(n), float(margin), _p(meta))
    return meta


def build_grid(mesh, n: int, margin: float):
    """Link SDF grid of one mesh: (values n^3 x-fastest, meta[10])."""
    v, t = _d(mesh.verts), np.ascontiguousarray(mesh.tris, np.int32)
    off = np.ascontiguousarray(mesh.comp_offsets, np.int32)
    vals = np.empty(int(n) ** 3)
    meta = np.empty(META_LEN)
    _load().oracle_build_grid(_p(v), int(v.shape[0]), _p(t), _p(off), int(off.shape[0] - 1),
                              int(n), float(margin), _p(vals), _p(meta))
    return vals, meta


def build_grids(meshes, n: int, margin: float):
    """All links: (list of value arrays, L x 10 meta)."""
    vals, metas = [], []
    for m in meshes:
        v, mt = build_grid(m, n, margin)
        vals.append(v)
        metas.append(mt)
    return vals, np.stack(metas)


# --------------------------------------------------------------------- FK

def fk(dh, base, q) -> np.ndarray:
    """World-from-link transforms, W x (dof+1) x 3 x 4."""
    dh, base = _d(dh, 6), _d(base)
    q = _d(np.atleast_2d(q))
    dof = dh.shape[0]
    if dof + 1 > _load().oracle_max_links():
        raise ValueError("too many links for the oracle")
    W = q.shape[0]
    out = np.empty((W, dof + 1, 3, 4))
    _load().oracle_fk(_p(dh), int(dof), _p(base), _p(q), int(W), _p(out))
    return out


# ------------------------------------------------------------------ lookup

def lookup(values, meta, p_loc) -> np.ndarray:
    """Interpolated link SDF at link-frame points (M x 3)."""
    vals, meta = _d(values), _d(meta)
    p = _d(np.atleast_2d(p_loc), 3)
    out = np.empty(p.shape[0])
    _load().oracle_lookup_many(_p(vals), _p(meta), _p(p), int(p.shape[0]), _p(out))
    return out


def _pack_grids(values, metas):
    L = len(values)
    offsets = np.zeros(L, dtype=np.int64)
    acc = 0
    for i, v in enumerate(values):
        offsets[i] = acc
        acc += int(np.asarray(v).size)
    flat = _d(np.concatenate([np.ravel(v) for v in values])) if L else np.zeros(0)
    return flat, offsets, _d(metas).reshape(L, META_LEN)


def check(dh, base, values, metas, q, points):
    """Per-waypoint (dist, argmin_link, argmin_point) -- the full oracle check."""
    dh, base = _d(dh, 6), _d(base)
    q = _d(q).reshape(-1, dh.shape[0])
    pts = _d(points).reshape(-1, 3)
    flat, offsets, metas = _pack_grids(values, metas)
    if metas.shape[0] != dh.shape[0] + 1:
        raise ValueError("need one grid per link (dof + 1)")
    W, N = q.shape[0], pts.shape[0]
    dist = np.empty(W)
    al = np.empty(W, np.int32)
    ap = np.empty(W, np.int32)
    _load().oracle_check(_p(dh), int(dh.shape[0]), _p(base), _p(flat), _p(offsets), _p(metas),
                         _p(q), int(W), _p(pts), int(N), _p(dist), _p(al), _p(ap))
    return dist, al, ap


def pair_values(dh, base, values, metas, q, points) -> np.ndarray:
    """Every (waypoint, link, point) interpolated distance, W x L x N."""
    dh, base = _d(dh, 6), _d(base)
    q = _d(q).reshape(-1, dh.shape[0])
    pts = _d(points).reshape(-1, 3)
    flat, offsets, metas = _pack_grids(values, metas)
    W, N, L = q.shape[0], pts.shape[0], dh.shape[0] + 1
    out = np.empty((W, L, N))
    _load().oracle_pair_values(_p(dh), int(dh.shape[0]), _p(base), _p(flat), _p(offsets),
                               _p(metas), _p(q), int(W), _p(pts), int(N), _p(out))
    return out


def build_grids_cached(meshes, n: int, margin: float, cache_dir: str | None = None):
    """``build_grids`` with an on-disk cache keyed by a hash of the meshes and grid
    parameters (the full-size brute-force build takes about a minute)."""
    import hashlib
    import tempfile
    h = hashlib.sha256()
    for m in meshes:
        for a in (np.ascontiguousarray(m.verts, np.float64), np.ascontiguousarray(m.tris, np.int32),
                  np.ascontiguousarray(m.comp_offsets, np.int32)):
            h.update(a.tobytes())
    h.update(np.array([n, margin], dtype=np.float64).tobytes())
    h.update(open(_SRC, "rb").read())
    d = cache_dir or os.path.join(tempfile.gettempdir(), "sdfcheck_oracle_grids")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, h.hexdigest()[:32] + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return list(z["values"]), z["metas"]
    vals, metas = build_grids(meshes, n, margin)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, values=np.stack(vals), metas=metas)
    os.replace(tmp, path)
    return vals, metas
