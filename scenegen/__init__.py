"""Seeded synthetic scene generators: arms, link meshes, trajectories, obstacle clouds.

This module produces INPUTS only.  It holds none of the distance-check arithmetic
(no signed distances, no forward kinematics, no interpolation), so both the FP64
oracle and the CUDA path can consume its output without sharing method code.

The paper's robot (DENSO VS-060, Sec. IV-C) and its Kinect v2 / RealSense recordings
(Sec. IV-C, IV-D) are not available, so every scene is synthetic with the paper's
scale: a 6-DoF serial arm with 7 link shapes (Sec. II-A), 300-500 waypoints along a
planned trajectory (Sec. IV-B, IV-C) and voxelised obstacle clouds (Sec. III-A,
IV-C).

Conventions
-----------
* Robot: standard Denavit-Hartenberg, revolute joints.  Row j of ``dh`` holds
  ``(a, alpha, d, theta_offset, q_min, q_max)`` of joint j+1.  Link 0 is the static
  base link (frame 0 = world), link j (1..dof) lives in DH frame j, so L = dof + 1.
* Meshes: float64 vertices in the link's own frame (metres), int32 triangles with
  counter-clockwise order seen from outside (outward normals), grouped into closed
  components by ``comp_offsets`` (triangle index where each component starts, plus
  the total as last entry).
* Points: float64 ``N x 3`` world coordinates (metres).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Mesh", "Scene", "gen_arm", "capsule_mesh", "uv_sphere_mesh", "box_mesh",
    "merge_meshes", "link_meshes", "spline_trajectory", "cloud_uniform",
    "cloud_humans", "make_scene", "SCENES",
]


@dataclasses.dataclass
class Mesh:
    verts: np.ndarray          # (V, 3) float64
    tris: np.ndarray           # (T, 3) int32
    comp_offsets: np.ndarray   # (C + 1,) int32: component c = tris[off[c]:off[c+1]]

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_components(self) -> int:
        return int(self.comp_offsets.shape[0] - 1)


@dataclasses.dataclass
class Scene:
    name: str
    dh: np.ndarray             # (dof, 6) float64
    base: np.ndarray           # (3, 4) float64, world-from-base transform
    meshes: list               # L meshes
    resolution: int            # grid nodes per axis
    margin: float              # metres added around each mesh's bounding box
    q: np.ndarray              # (W, dof) float64
    points: np.ndarray         # (N, 3) float64

    @property
    def dof(self) -> int:
        return int(self.dh.shape[0])

    @property
    def n_links(self) -> int:
        return len(self.meshes)


# --------------------------------------------------------------------------- arms

def gen_arm(rng: np.random.Generator, dof: int, length_range=(0.1, 0.4)) -> np.ndarray:
    """Random serial arm: each link offset lies along DH ``a`` or ``d``.

    Link length uniform in ``length_range`` metres, twist from {-pi/2, 0, pi/2},
    joint limits symmetric with half-range uniform in [120, 170] degrees.
    """
    dh = np.zeros((dof, 6), dtype=np.float64)
    for j in range(dof):
        length = rng.uniform(*length_range)
        along_a = rng.random() < 0.5
        alpha = rng.choice([-math.pi / 2, 0.0, math.pi / 2])
        theta_off = rng.uniform(-math.pi, math.pi)
        lim = math.radians(rng.uniform(120.0, 170.0))
        dh[j] = (length if along_a else 0.0, alpha, 0.0 if along_a else length,
                 theta_off, -lim, lim)
    return dh


# ------------------------------------------------------------------------- meshes

def _orthonormal_frame(axis: np.ndarray):
    axis = axis / np.linalg.norm(axis)
    helper = np.array([1.0, 0.0, 0.0]) if abs(axis[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(axis, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(axis, e1)
    return axis, e1, e2


def _ring_strip(rings, poles_first, pole_last):
    """Triangles joining a pole, a list of vertex rings (index arrays) and a pole."""
    tris = []
    m = len(rings[0])
    r0 = rings[0]
    for k in range(m):
        tris.append((poles_first, r0[k], r0[(k + 1) % m]))
    for a, b in zip(rings[:-1], rings[1:]):
        for k in range(m):
            k1 = (k + 1) % m
            tris.append((a[k], b[k], b[k1]))
            tris.append((a[k], b[k1], a[k1]))
    rl = rings[-1]
    for k in range(m):
        tris.append((pole_last, rl[(k + 1) % m], rl[k]))
    return tris


def _orient_outward(verts, tris, inside_of):
    """Flip triangles whose normal points toward the interior reference point(s)."""
    tris = np.asarray(tris, dtype=np.int64)
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    out = cen - inside_of(cen)
    flip = np.einsum("ij,ij->i", nrm, out) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris.astype(np.int32)


def capsule_mesh(p0, p1, radius: float, n_lon: int, n_lat: int) -> Mesh:
    """Closed capsule around segment p0-p1: two hemispheres of ``n_lat`` rings each.

    All vertices lie on the exact capsule surface; ``4 * n_lon * n_lat`` triangles.
    """
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    seg = p1 - p0
    if np.linalg.norm(seg) < 1e-9:
        return uv_sphere_mesh(p0, radius, n_lon, 2 * n_lat)
    u, e1, e2 = _orthonormal_frame(seg)
    verts = []
    phis = 2.0 * math.pi * np.arange(n_lon) / n_lon

    def ring(center, polar, direction):
        # polar angle measured from the cap's pole direction
        s, c = math.sin(polar), math.cos(polar)
        idx = []
        for ph in phis:
            v = center + radius * (c * direction + s * (math.cos(ph) * e1 + math.sin(ph) * e2))
            idx.append(len(verts))
            verts.append(v)
        return idx

    verts.append(p1 + radius * u)
    top_pole = 0
    rings = []
    for k in range(1, n_lat + 1):
        rings.append(ring(p1, (math.pi / 2) * k / n_lat, u))
    for k in range(n_lat, 0, -1):
        rings.append(ring(p0, (math.pi / 2) * k / n_lat, -u))
    verts.append(p0 - radius * u)
    bottom_pole = len(verts) - 1
    verts = np.asarray(verts)
    tris = _ring_strip(rings, top_pole, bottom_pole)

    def axis_point(x):
        t = np.clip((x - p0) @ seg / (seg @ seg), 0.0, 1.0)
        return p0 + t[:, None] * seg

    tris = _orient_outward(verts, tris, axis_point)
    return Mesh(verts, tris, np.array([0, len(tris)], dtype=np.int32))


def uv_sphere_mesh(center, radius: float, n_lon: int, n_lat: int) -> Mesh:
    """Closed UV sphere, ``n_lat - 1`` rings between the poles; vertices on the sphere."""
    center = np.asarray(center, dtype=np.float64)
    verts = [center + np.array([0.0, 0.0, radius])]
    rings = []
    for k in range(1, n_lat):
        th = math.pi * k / n_lat
        idx = []
        for m in range(n_lon):
            ph = 2.0 * math.pi * m / n_lon
            idx.append(len(verts))
            verts.append(center + radius * np.array([math.sin(th) * math.cos(ph),
                                                     math.sin(th) * math.sin(ph),
                                                     math.cos(th)]))
        rings.append(idx)
    verts.append(center - np.array([0.0, 0.0, radius]))
    verts = np.asarray(verts)
    tris = _ring_strip(rings, 0, len(verts) - 1)
    tris = _orient_outward(verts, tris, lambda x: np.broadcast_to(center, x.shape))
    return Mesh(verts, tris, np.array([0, len(tris)], dtype=np.int32))


def box_mesh(center, half, subdiv: int = 1) -> Mesh:
    """Closed axis-aligned box, each face split into ``subdiv x subdiv`` quads."""
    center = np.asarray(center, dtype=np.float64)
    half = np.asarray(half, dtype=np.float64)
    verts, tris = [], []
    key = {}
    g = np.linspace(-1.0, 1.0, subdiv + 1)

    def vid(p):
        k = tuple(np.round(p, 12))
        if k not in key:
            key[k] = len(verts)
            verts.append(center + p * half)
        return key[k]

    for axis in range(3):
        for sign in (-1.0, 1.0):
            a1, a2 = [x for x in range(3) if x != axis]
            for i in range(subdiv):
                for j in range(subdiv):
                    quad = []
                    for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = np.zeros(3)
                        p[axis] = sign
                        p[a1] = g[i + di]
                        p[a2] = g[j + dj]
                        quad.append(vid(p))
                    tris.append((quad[0], quad[1], quad[2]))
                    tris.append((quad[0], quad[2], quad[3]))
    verts = np.asarray(verts)
    tris = _orient_outward(verts, tris, lambda x: np.broadcast_to(center, x.shape))
    return Mesh(verts, tris, np.array([0, len(tris)], dtype=np.int32))


def merge_meshes(parts) -> Mesh:
    """Union of closed meshes kept as separate components (no boolean surgery)."""
    verts, tris, offs = [], [], [0]
    base = 0
    for m in parts:
        verts.append(m.verts)
        tris.append(m.tris + base)
        base += m.verts.shape[0]
        offs.append(offs[-1] + m.n_tris)
    return Mesh(np.concatenate(verts), np.concatenate(tris).astype(np.int32),
                np.asarray(offs, dtype=np.int32))


def _prev_joint_in_frame(a, alpha, d):
    """Origin of DH frame j-1 expressed in frame j (independent of the joint angle)."""
    return np.array([-a, -d * math.sin(alpha), -d * math.cos(alpha)])


def link_meshes(rng: np.random.Generator, dh: np.ndarray, kind: str,
                n_lon: int, n_lat: int, box_subdiv: int = 2) -> list:
    """One mesh per link: a capsule along the link (plus a joint housing box).

    kind = "capsule": capsule only; "capsule_box": capsule plus an axis-aligned box
    around the joint at the frame origin (a two-component union).
    """
    meshes = []
    r_base = rng.uniform(0.06, 0.09)
    spans = [(np.array([0.0, 0.0, -0.15]), np.zeros(3), r_base)]
    for j in range(dh.shape[0]):
        a, alpha, d = dh[j, 0], dh[j, 1], dh[j, 2]
        spans.append((_prev_joint_in_frame(a, alpha, d), np.zeros(3), rng.uniform(0.04, 0.08)))
    for (p0, p1, r) in spans:
        cap = capsule_mesh(p0, p1, r, n_lon, n_lat)
        if kind == "capsule":
            meshes.append(cap)
        elif kind == "capsule_box":
            half = np.array([1.15 * r, 1.15 * r, 1.4 * r])
            meshes.append(merge_meshes([cap, box_mesh(np.zeros(3), half, box_subdiv)]))
        else:
            raise ValueError(kind)
    return meshes


# ------------------------------------------------------------------- trajectories

def spline_trajectory(rng: np.random.Generator, dh: np.ndarray, n_via: int, W: int,
                      limit_fraction: float = 0.9) -> np.ndarray:
    """Clamped cubic spline (zero end velocity, uniform knots) through ``n_via``
    random in-limit configurations, sampled at W points including both ends."""
    from scipy.interpolate import CubicSpline
    dof = dh.shape[0]
    lo = dh[:, 4] * limit_fraction
    hi = dh[:, 5] * limit_fraction
    via = rng.uniform(lo, hi, size=(n_via, dof))
    if W == 0:
        return np.zeros((0, dof))
    knots = np.linspace(0.0, 1.0, n_via)
    spl = CubicSpline(knots, via, axis=0, bc_type="clamped")
    q = spl(np.linspace(0.0, 1.0, W))
    return np.clip(q, dh[:, 4], dh[:, 5])


# -------------------------------------------------------------------------- clouds

def cloud_uniform(rng: np.random.Generator, N: int, side: float = 2.0,
                  center=(0.0, 0.0, 0.0)) -> np.ndarray:
    return rng.uniform(-side / 2, side / 2, size=(N, 3)) + np.asarray(center)


def _capsule_contains(x, p0, p1, r):
    seg = p1 - p0
    t = np.clip((x - p0) @ seg / (seg @ seg), 0.0, 1.0)
    return np.linalg.norm(x - (p0 + t[:, None] * seg), axis=1) <= r


def human_capsules(rng: np.random.Generator, dist_range=(0.2, 1.5),
                   torso_r=0.3, torso_len=0.5, limb_r=0.06, limb_len=0.6):
    """A standing human-like cluster: a vertical torso capsule and four limbs.

    The torso surface is ``dist_range`` metres (horizontally) from the base axis.
    Returns a list of (p0, p1, r) capsules in world coordinates.
    """
    rho = rng.uniform(*dist_range) + torso_r
    az = rng.uniform(-math.pi, math.pi)
    yaw = rng.uniform(-math.pi, math.pi)
    z0 = rng.uniform(-0.3, 0.3)
    c = np.array([rho * math.cos(az), rho * math.sin(az), z0])
    rot = np.array([[math.cos(yaw), -math.sin(yaw), 0.0],
                    [math.sin(yaw), math.cos(yaw), 0.0],
                    [0.0, 0.0, 1.0]])
    caps = [(np.array([0.0, 0.0, 0.0]), np.array([0.0, 0.0, torso_len]), torso_r)]
    for side in (-1.0, 1.0):
        shoulder = np.array([side * (torso_r + limb_r), 0.0, torso_len])
        el = rng.uniform(-0.6 * math.pi, 0.6 * math.pi)
        azl = rng.uniform(-math.pi, math.pi)
        dirv = np.array([math.cos(el) * math.cos(azl), math.cos(el) * math.sin(azl), math.sin(el)])
        caps.append((shoulder, shoulder + limb_len * dirv, limb_r))
        hip = np.array([side * 0.15, 0.0, -torso_r * 0.5])
        caps.append((hip, hip + np.array([0.0, 0.0, -limb_len]), limb_r))
    return [(c + rot @ p0, c + rot @ p1, r) for (p0, p1, r) in caps]


def human_voxels(rng: np.random.Generator, n_clusters: int = 3, voxel: float = 0.02, clusters=None) -> np.ndarray:
    """Integer cells of the occupied ``voxel``-sized voxels of ``n_clusters``
    human-like clusters (unique, unordered)."""
    if clusters is None:
        clusters = [human_capsules(rng) for _ in range(n_clusters)]
    keys = []
    for caps in clusters:
        lo = np.min([np.minimum(p0, p1) - r for (p0, p1, r) in caps], axis=0)
        hi = np.max([np.maximum(p0, p1) + r for (p0, p1, r) in caps], axis=0)
        ilo = np.floor(lo / voxel).astype(np.int64)
        ihi = np.ceil(hi / voxel).astype(np.int64)
        axes = [np.arange(ilo[a], ihi[a] + 1) for a in range(3)]
        gi = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
        x = (gi + 0.5) * voxel
        occ = np.zeros(x.shape[0], dtype=bool)
        for (p0, p1, r) in caps:
            occ |= _capsule_contains(x, p0, p1, r)
        keys.append(gi[occ])
    return np.unique(np.concatenate(keys), axis=0)


def sample_voxels(rng: np.random.Generator, cells: np.ndarray, N: int, voxel: float = 0.02,
                  order: str = "voxel") -> np.ndarray:
    """N voxel centres drawn without replacement from integer cells.

    order = "voxel": sorted by linear voxel index (x fastest), the order in which a
    voxeliser emits occupied cells; "random": shuffled.
    """
    if N > cells.shape[0]:
        raise ValueError(f"only {cells.shape[0]} occupied voxels, {N} requested")
    pick = rng.choice(cells.shape[0], size=N, replace=False)
    cells = cells[pick]
    if order == "voxel" and N > 0:
        off = cells - cells.min(axis=0)
        ext = off.max(axis=0) + 1
        lin = off[:, 0] + ext[0] * (off[:, 1] + ext[1] * off[:, 2])
        cells = cells[np.argsort(lin, kind="stable")]
    elif order not in ("voxel", "random"):
        raise ValueError(order)
    return (cells + 0.5) * voxel


def cloud_humans(rng: np.random.Generator, N: int, n_clusters: int = 3, voxel: float = 0.02,
                 order: str = "voxel", clusters=None) -> np.ndarray:
    """N occupied ``voxel``-sized voxel centres of ``n_clusters`` human-like
    clusters, sampled without replacement (see ``sample_voxels`` for the order)."""
    cells = human_voxels(rng, n_clusters, voxel, clusters)
    return sample_voxels(rng, cells, N, voxel, order)


# ------------------------------------------------------------------------ configs

SCENES = {
    # 6-DoF, 7 capsule links of 512 triangles, 32^3 grids, 50 waypoints through
    # 3 configurations, 1,000 points uniform in a 2 m cube.
    "tiny": dict(seed=1, dof=6, kind="capsule", n_lon=16, n_lat=8, resolution=32,
                 margin=0.05, n_via=3, W=50, cloud="uniform", N=1000),
    # Same generator, capsule+box links of 1,968 triangles, 96^3 grids, 500
    # waypoints through 5 configurations, 20,000 2 cm voxel centres of 3 humans.
    "paper": dict(seed=2, dof=6, kind="capsule_box", n_lon=32, n_lat=15, resolution=96,
                  margin=0.05, n_via=5, W=500, cloud="humans", N=20000),
}


def make_scene(name: str, **override) -> Scene:
    """Build one of the named scenes ("tiny", "paper"); keyword overrides allowed
    (e.g. ``W``, ``N``, ``resolution``, ``order``)."""
    cfg = dict(SCENES[name])
    cfg.update(override)
    rng = np.random.default_rng(cfg["seed"])
    dh = gen_arm(rng, cfg["dof"])
    meshes = link_meshes(rng, dh, cfg["kind"], cfg["n_lon"], cfg["n_lat"])
    q = spline_trajectory(rng, dh, cfg["n_via"], cfg["W"])
    if cfg["cloud"] == "uniform":
        pts = cloud_uniform(rng, cfg["N"])
    else:
        pts = cloud_humans(rng, cfg["N"], order=cfg.get("order", "voxel"))
    base = np.hstack([np.eye(3), np.zeros((3, 1))])
    return Scene(name, dh, base, meshes, cfg["resolution"], cfg["margin"], q, pts)


# ------------------------------------------------------------ batched workload

@dataclasses.dataclass
class BatchedScene:
    arms: list                 # Scene per arm model (meshes, grid parameters, DH); q/points unused
    instances: list            # (arm index, q (W x dof), points (N x 3))


def make_batched(seed: int = 3, n: int = 64, W_range=(50, 1000), N_range=(1000, 100000),
                 resolution: int = 96, layouts: int = 8, order: str = "voxel") -> BatchedScene:
    """Independent checks of uneven sizes for one batched launch: a pool of two arm
    models (6- and 7-DoF, capsule+box links, ``resolution``^3 grids), trajectories of
    W ~ U(W_range) waypoints through 5 configurations, clouds of N log-uniform in
    N_range points drawn from a pool of ``layouts`` three-human voxel layouts."""
    rng = np.random.default_rng(seed)
    arms = []
    for dof in (6, 7):
        dh = gen_arm(rng, dof)
        meshes = link_meshes(rng, dh, "capsule_box", 32, 15)
        base = np.hstack([np.eye(3), np.zeros((3, 1))])
        arms.append(Scene(f"arm{dof}", dh, base, meshes, resolution, 0.05, np.zeros((0, dof)),
                          np.zeros((0, 3))))
    pool = [human_voxels(rng) for _ in range(layouts)]
    insts = []
    for i in range(n):
        a = int(rng.integers(0, 2))
        W = int(rng.integers(W_range[0], W_range[1] + 1))
        N = int(round(math.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1])))))
        cells = pool[int(rng.integers(0, layouts))]
        N = min(N, cells.shape[0])
        q = spline_trajectory(rng, arms[a].dh, 5, W)
        insts.append((a, q, sample_voxels(rng, cells, N, order=order)))
    return BatchedScene(arms, insts)


# ------------------------------------------------------------- serving workload

def drifting_clouds(seed: int = 5, cycles: int = 250, N_range=(5000, 80000), sigma: float = 0.005,
                    voxel: float = 0.02, order: str = "voxel"):
    """Clouds for a control-cycle stream: three human clusters whose positions take
    a Gaussian random walk (``sigma`` metres per axis per cycle, so a mean step of
    sigma * sqrt(8 / pi), about 0.8 cm), voxelised at ``voxel`` and sampled to N ~ U(N_range)
    points each cycle."""
    rng = np.random.default_rng(seed)
    clusters = [human_voxels(rng, 1, voxel) for _ in range(3)]
    offs = np.zeros((3, 3))
    out = []
    for _ in range(cycles):
        offs += rng.normal(0.0, sigma, size=(3, 3))
        shift = np.round(offs / voxel).astype(np.int64)
        cells = np.unique(np.concatenate([c + shift[i] for i, c in enumerate(clusters)]), axis=0)
        N = min(int(rng.integers(N_range[0], N_range[1] + 1)), cells.shape[0])
        out.append(sample_voxels(rng, cells, N, voxel, order).astype(np.float32))
    return out


# ------------------------------------------------------------ surrogate weights

MLP_HIDDEN = 128
MLP_PARAMS = MLP_HIDDEN * 3 + MLP_HIDDEN + 2 * (MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN) + MLP_HIDDEN + 1


def mlp_init(seed: int, links: int) -> np.ndarray:
    """Initial parameters of the per-link surrogate networks, [links, MLP_PARAMS] FP32:
    every weight and bias of a layer uniform in +-1/sqrt(fan_in), in the parameter
    order W1[128][3], b1, W2[128][128], b2, W3[128][128], b3, w4[128], b4."""
    rng = np.random.default_rng(seed)
    H = MLP_HIDDEN
    out = np.empty((links, MLP_PARAMS), dtype=np.float32)
    for l in range(links):
        parts = []
        for n, fan in ((H * 3, 3), (H, 3), (H * H, H), (H, H), (H * H, H), (H, H), (H, H), (1, H)):
            b = 1.0 / math.sqrt(fan)
            parts.append(rng.uniform(-b, b, n))
        out[l] = np.concatenate(parts)
    return out
