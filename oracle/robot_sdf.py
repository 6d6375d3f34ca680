"""FP64 CPU oracle for the paper's own formulation: Robot SDFs on an environment
voxel grid (test infrastructure; only tests, smoke() and bench.py's CPU leg use it).

Sec. III-A: the environment is a voxel grid; for every configuration each Link SDF
is transformed into the environment and aligned with its voxels (the Euclidean
transformation of Eq. (4) and the sub-voxel shift of Eq. (1)-(3)), the Robot SDF
of the configuration is the minimum over links per voxel, and at runtime the
obstacles are voxelised and the Robot SDF is read at the occupied voxels, the
minimum per configuration being the distance.  Transforming a link grid so that
its samples fall on environment voxel centres is the same as evaluating the link
SDF at each voxel centre mapped into the link frame, which is what this oracle
does (trilinear interpolation with the out-of-box rule, as the grid path).

Only the voxels inside a link's block are written for that link (Sec. III-B,
"grids in sphere"): the voxels whose centres lie within radius
R_link + reach + sqrt(3) r_e / 2 of the link's bounding-sphere centre, where reach
is the distance range the caller wants covered.  A voxel that no block covers
holds +inf.

Environment grid: origin o (lower corner), voxel edge r_e, dims (nx, ny, nz);
voxel (i, j, k) covers o + [i, i+1) r_e etc. (the index taken in single precision,
see voxel_of), its centre o + (i + 1/2) r_e, and its linear index is
i + nx (j + ny k).  A point outside the grid occupies no voxel.

Parity status: pinned by reduction to the per-point check (every voxel in every
block gives oracle.check at the occupied voxel centres) and by hand-computed
voxelisations (tests/test_oracle_robot_sdf.py).
"""
from __future__ import annotations

import numpy as np

import oracle


def voxel_of(points, origin, voxel, dims):
    """Linear voxel index of each point, -1 outside the grid or non-finite.  The
    index is an integer decided by floating point, so it is taken in single
    precision as the GPU takes it: floor((p - o) * fl32(1 / r)), each operation
    rounded to float32, no fused multiply-add."""
    p32 = np.asarray(points, dtype=np.float32).reshape(-1, 3)
    o32 = np.asarray(origin, dtype=np.float32)
    inv = np.float32(1.0 / float(voxel))
    with np.errstate(invalid="ignore", over="ignore"):
        p = ((p32 - o32).astype(np.float32) * inv).astype(np.float32)
        ijk = np.floor(p.astype(np.float64))
    ok = np.all(np.isfinite(ijk), axis=1)
    d = np.asarray(dims)
    ok &= np.all((ijk >= 0) & (ijk < d), axis=1)
    ijk = np.where(ok[:, None], ijk, 0).astype(np.int64)
    lin = ijk[:, 0] + d[0] * (ijk[:, 1] + d[1] * ijk[:, 2])
    return np.where(ok, lin, -1)


def occupied(points, origin, voxel, dims):
    """Sorted linear indices of the voxels that hold at least one point."""
    v = voxel_of(points, origin, voxel, dims)
    return np.unique(v[v >= 0])


def voxel_centres(lin, origin, voxel, dims):
    lin = np.asarray(lin, dtype=np.int64)
    nx, ny = int(dims[0]), int(dims[1])
    i = lin % nx
    j = (lin // nx) % ny
    k = lin // (nx * ny)
    return np.asarray(origin, dtype=np.float64) + (np.stack([i, j, k], axis=1) + 0.5) * voxel


def robot_sdf_values(dh, base, values, metas, q, voxels, origin, voxel, dims, reach):
    """Robot SDF at the given voxels for every configuration: [W, len(voxels)]."""
    T = oracle.fk(dh, base, q)                        # [W, L, 3, 4] world-from-link
    W, L = T.shape[0], T.shape[1]
    x = voxel_centres(voxels, origin, voxel, dims)    # [V, 3]
    out = np.full((W, x.shape[0]), np.inf)
    pad = np.sqrt(3.0) * voxel / 2.0
    for w in range(W):
        for l in range(L):
            meta = np.asarray(metas[l], dtype=np.float64)
            R, t = T[w, l, :, :3], T[w, l, :, 3]
            c_world = R @ meta[5:8] + t
            rho = meta[8] + reach + pad
            inside = np.linalg.norm(x - c_world, axis=1) <= rho
            if not np.any(inside):
                continue
            p_loc = (x[inside] - t) @ R
            g = oracle.lookup(values[l], meta, p_loc)
            out[w, inside] = np.minimum(out[w, inside], g)
    return out


def check(dh, base, values, metas, q, points, origin, voxel, dims, reach):
    """Per configuration: the minimum Robot SDF value over the occupied voxels and
    the voxel attaining it (smallest index on ties); +inf and -1 when no occupied
    voxel lies in a block."""
    occ = occupied(points, origin, voxel, dims)
    W = np.atleast_2d(q).shape[0]
    if occ.size == 0:
        return np.full(W, np.inf), np.full(W, -1, dtype=np.int64)
    v = robot_sdf_values(dh, base, values, metas, q, occ, origin, voxel, dims, reach)
    i = np.argmin(v, axis=1)
    d = v[np.arange(W), i]
    return d, np.where(np.isfinite(d), occ[i], -1)
