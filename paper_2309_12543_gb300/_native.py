"""ctypes binding of libsdfcheck (the C ABI in include/sdfcheck.h).

Argument marshalling only: every step of the distance check runs in the CUDA
library.  Device buffers are passed as torch CUDA tensors (or raw integer
addresses); host buffers as numpy arrays.  If the compiled library is missing the
import fails with an error -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsdfcheck.so")

SDF_OK = 0
SDF_ERR_INVALID_ARG = -1
SDF_ERR_OOM = -2
SDF_ERR_CUDA = -3
SDF_ERR_TIMEOUT = -4
SDF_ERR_UNSUPPORTED = -5
SDF_ERR_NONFINITE = -6
SDF_PENDING = 1
SDF_MAX_LINKS = 16
SDF_MAX_POINTS = 16777215
SDF_NOALLOC_MAX_POINTS = 32768
SDF_MAX_BATCH = 128
SDF_MLP_HIDDEN = 128
SDF_MLP_PARAMS = 33665
SDF_MLP_BATCH = 128

SDF_OPT_CULL = 1
SDF_OPT_POINT_STRIDE = 2
SDF_OPT_WAYPOINTS_PER_BLOCK = 3
SDF_OPT_TILE_BATCH = 4
SDF_OPT_TIME_KERNELS = 6
SDF_OPT_STATS = 7
SDF_OPT_BLOCK_WARPS = 8
SDF_OPT_WAIT_POLLS = 9
SDF_OPT_TEX3D = 10
SDF_OPT_SORT_CTAS = 11
SDF_KERNEL_PREP = 0
SDF_KERNEL_CHECK = 1

ERROR_NAMES = {0: "SDF_OK", -1: "SDF_ERR_INVALID_ARG", -2: "SDF_ERR_OOM", -3: "SDF_ERR_CUDA",
               -4: "SDF_ERR_TIMEOUT", -5: "SDF_ERR_UNSUPPORTED", -6: "SDF_ERR_NONFINITE"}


class SdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class sdf_mesh(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int32),
                ("tris", ctypes.c_void_p), ("n_tris", ctypes.c_int32),
                ("n_components", ctypes.c_int32), ("comp_tri_offsets", ctypes.c_void_p)]


class sdf_dh(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("a", "alpha", "d", "theta_offset", "q_min", "q_max")]


class sdf_check_request(ctypes.Structure):
    _fields_ = [("robot", ctypes.c_void_p), ("q_dev", ctypes.c_void_p), ("W", ctypes.c_int32),
                ("points_dev", ctypes.c_void_p), ("N", ctypes.c_int32), ("dist_dev", ctypes.c_void_p),
                ("argmin_link_dev", ctypes.c_void_p), ("argmin_point_dev", ctypes.c_void_p),
                ("mask_dev", ctypes.c_void_p)]


class sdf_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("memory_budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_waypoints", ctypes.c_int32), ("max_points", ctypes.c_int32),
                ("max_dof", ctypes.c_int32), ("batch_window_us", ctypes.c_int32)]


class sdf_env_grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float), ("dims", ctypes.c_int32 * 3),
                ("reach", ctypes.c_float)]


class sdf_grid_meta(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("n", ctypes.c_int32),
                ("center", ctypes.c_float * 3), ("radius", ctypes.c_float), ("margin", ctypes.c_float)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2309_12543_gb300.build.build() "
                          "(nvcc for sm_103a) -- there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sigs = {
        "sdf_ctx_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
        "sdf_ctx_destroy": (None, [P]),
        "sdf_ctx_set_stream": (ctypes.c_int, [P, P]),
        "sdf_last_error": (ctypes.c_char_p, [P]),
        "sdf_ctx_set_option": (ctypes.c_int, [P, i32, i64]),
        "sdf_ctx_get_option": (ctypes.c_int, [P, i32, ctypes.POINTER(i64)]),
        "sdf_ctx_synchronize": (ctypes.c_int, [P]),
        "sdf_ctx_stats": (ctypes.c_int, [P, P, i32, i32]),
        "sdf_measure_gather": (ctypes.c_int, [P, P, P, P]),
        "sdf_surrogate_create": (ctypes.c_int, [P, P, P, P]),
        "sdf_surrogate_destroy": (None, [P]),
        "sdf_surrogate_params": (ctypes.c_int, [P, P, P]),
        "sdf_surrogate_sample": (ctypes.c_int, [P, P, i32, i64, i32, ctypes.c_float, ctypes.c_uint64, P, P, P]),
        "sdf_surrogate_grad": (ctypes.c_int, [P, P, i32, P, P, P, P]),
        "sdf_surrogate_train": (ctypes.c_int, [P, P, P, P, i64, i64, i32, ctypes.c_float, P]),
        "sdf_surrogate_eval": (ctypes.c_int, [P, P, i32, P, i32, P]),
        "sdf_surrogate_error": (ctypes.c_int, [P, P, i32, i64, i32, ctypes.c_float, ctypes.c_uint64, P, P]),
        "check_trajectory_surrogate": (ctypes.c_int, [P, P, P, P, i32, P, i32, ctypes.c_float, ctypes.c_float,
                                                      P, P, P, P, P]),
        "sdf_server_set_surrogate": (ctypes.c_int, [P, P, ctypes.c_float, ctypes.c_float]),
        "check_trajectory_robot_sdf": (ctypes.c_int, [P, P, P, P, i32, P, i32, P, P]),
        "sdf_ctx_last_kernel_ms": (ctypes.c_int, [P, i32, ctypes.POINTER(ctypes.c_float)]),
        "sdf_build_grids": (ctypes.c_int, [P, P, i32, i32, ctypes.c_float, ctypes.POINTER(P)]),
        "sdf_grids_upload": (ctypes.c_int, [P, P, P, i32, ctypes.POINTER(P)]),
        "sdf_grids_download": (ctypes.c_int, [P, P, P, P]),
        "sdf_grids_info": (ctypes.c_int, [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "sdf_grids_destroy": (None, [P]),
        "sdf_robot_create": (ctypes.c_int, [P, P, i32, P, P, ctypes.POINTER(P)]),
        "sdf_robot_destroy": (None, [P]),
        "sdf_forward_kinematics": (ctypes.c_int, [P, P, P, i32, P]),
        "check_trajectory": (ctypes.c_int, [P, P, P, i32, P, i32, P, P, P]),
        "check_trajectory_host": (ctypes.c_int, [P, P, P, i32, P, i32, P, P, P]),
        "check_trajectory_noalloc": (ctypes.c_int, [P, P, P, i32, P, i32, P, P, P, P]),
        "check_batch": (ctypes.c_int, [P, P, i32]),
        "sdf_autotune": (ctypes.c_int, [P, P, i32, i32, P, P, P]),
        "sdf_server_create": (ctypes.c_int, [P, ctypes.POINTER(P)]),
        "sdf_server_destroy": (None, [P]),
        "sdf_server_set_cloud": (ctypes.c_int, [P, P, i32]),
        "sdf_server_submit": (ctypes.c_int, [P, P, P, i32, ctypes.POINTER(ctypes.c_uint64)]),
        "sdf_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, i64, P, P, P, ctypes.POINTER(ctypes.c_double)]),
        "sdf_server_stats": (ctypes.c_int, [P, P, i32, i32]),
        "sdf_ctx_reserve": (ctypes.c_int, [P, i64, i64, i64, i32]),
        "sdf_debug_fail_alloc": (ctypes.c_int, [i64]),
        "sdf_debug_alloc_live": (ctypes.c_int, [P, P, P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# the symbols include/sdfcheck.h declares (tests check the export table against it)
EXPORTED = ("sdf_ctx_create", "sdf_ctx_destroy", "sdf_ctx_set_stream", "sdf_last_error",
            "sdf_ctx_set_option", "sdf_ctx_get_option", "sdf_ctx_synchronize",
            "sdf_ctx_last_kernel_ms", "sdf_ctx_stats", "sdf_build_grids", "sdf_grids_upload", "sdf_grids_download",
            "sdf_grids_info", "sdf_grids_destroy", "sdf_robot_create", "sdf_robot_destroy",
            "sdf_forward_kinematics", "check_trajectory", "check_trajectory_host",
            "check_trajectory_noalloc", "check_batch", "sdf_ctx_reserve", "sdf_autotune",
            "sdf_server_create", "sdf_server_destroy", "sdf_server_set_cloud", "sdf_server_submit",
            "sdf_server_poll", "sdf_server_stats", "sdf_measure_gather", "sdf_surrogate_create",
            "sdf_surrogate_destroy", "sdf_surrogate_params", "sdf_surrogate_sample", "sdf_surrogate_grad",
            "sdf_surrogate_train", "sdf_surrogate_eval", "sdf_surrogate_error", "check_trajectory_surrogate",
            "sdf_server_set_surrogate", "check_trajectory_robot_sdf", "sdf_debug_fail_alloc",
            "sdf_debug_alloc_live")


def _ptr(x) -> int:
    """Device address of a torch tensor (or an int), host address of a numpy array."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(type(x))


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Context:
    """Owns an sdf_ctx: device, stream binding, scratch and options."""

    def __init__(self, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        rc = lib.sdf_ctx_create(ctypes.byref(h), int(device), _stream_handle(stream))
        if rc != SDF_OK:
            raise SdfError(rc, "sdf_ctx_create failed")
        self.handle = h
        self.device = device

    def _check(self, rc: int, what: str):
        if rc != SDF_OK:
            raise SdfError(rc, f"{what}: {lib.sdf_last_error(self.handle).decode()}")

    def set_stream(self, stream):
        self._check(lib.sdf_ctx_set_stream(self.handle, _stream_handle(stream)), "set_stream")

    def set_option(self, key: int, value: int):
        self._check(lib.sdf_ctx_set_option(self.handle, int(key), int(value)), "set_option")

    def get_option(self, key: int) -> int:
        v = ctypes.c_int64()
        self._check(lib.sdf_ctx_get_option(self.handle, int(key), ctypes.byref(v)), "get_option")
        return int(v.value)

    def synchronize(self) -> int:
        """Wait for the stream; return the device status code (does not raise)."""
        return int(lib.sdf_ctx_synchronize(self.handle))

    def last_error(self) -> str:
        return lib.sdf_last_error(self.handle).decode()

    STAT_NAMES = ("pairs", "seed_lookups", "super_tests", "super_pass", "tile_tests", "tile_pass",
                  "point_tests", "lookups", "list_overflow", "blocks", "ns_fk", "ns_seed", "ns_cull",
                  "ns_points", "ns_block", "ns_block_max", "ns_span", "_17", "_18", "sur_ns_cta", "ns_sort_box",
                  "ns_sort_hist", "ns_sort_scan", "ns_sort_scatter", "ns_sort_tiles", "ns_sort_supers",
                  "sur_seed_queries", "sur_queries", "sur_ns_produce", "sur_ns_eval", "sur_ns_list",
                  "sur_ns_cta_max")

    def stats(self, reset: bool = False) -> dict:
        """Counters accumulated while SDF_OPT_STATS is on (see sdfcheck.h)."""
        out = np.zeros(32, dtype=np.int64)
        self._check(lib.sdf_ctx_stats(self.handle, _ptr(out), 32, int(reset)), "sdf_ctx_stats")
        return {k: int(v) for k, v in zip(self.STAT_NAMES, out) if not k.startswith("_")}

    def last_kernel_ms(self, kernel: int = 1) -> float:
        """Device ms of SDF_KERNEL_PREP (0) or SDF_KERNEL_CHECK (1) of the last check."""
        v = ctypes.c_float()
        self._check(lib.sdf_ctx_last_kernel_ms(self.handle, int(kernel), ctypes.byref(v)), "last_kernel_ms")
        return float(v.value)

    def close(self):
        if getattr(self, "handle", None):
            lib.sdf_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grids:
    """Owns an sdf_grids handle (device Link SDFs + metadata)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle
        nl, n = ctypes.c_int32(), ctypes.c_int32()
        lib.sdf_grids_info(handle, ctypes.byref(nl), ctypes.byref(n))
        self.n_links, self.resolution = int(nl.value), int(n.value)

    def download(self):
        """(values float32 [L, n^3], meta list of dicts)."""
        L, n = self.n_links, self.resolution
        vals = np.empty((L, n ** 3), dtype=np.float32)
        metas = (sdf_grid_meta * L)()
        self.ctx._check(lib.sdf_grids_download(self.ctx.handle, self.handle, _ptr(vals),
                                               ctypes.addressof(metas)), "sdf_grids_download")
        return vals, [meta_to_dict(m) for m in metas]

    def close(self):
        if getattr(self, "handle", None):
            lib.sdf_grids_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def meta_to_dict(m: sdf_grid_meta) -> dict:
    return dict(origin=np.array(m.origin[:], dtype=np.float32), h=float(m.h), n=int(m.n),
                center=np.array(m.center[:], dtype=np.float32), radius=float(m.radius),
                margin=float(m.margin))


def sdf_build_grids(ctx: Context, meshes, resolution: int, margin: float) -> Grids:
    """meshes: objects with verts (V x 3), tris (T x 3) and comp_offsets (C + 1)."""
    keep = []
    arr = (sdf_mesh * len(meshes))()
    for i, m in enumerate(meshes):
        v = np.ascontiguousarray(m.verts, dtype=np.float32)
        t = np.ascontiguousarray(m.tris, dtype=np.int32)
        off = np.ascontiguousarray(m.comp_offsets, dtype=np.int32)
        keep += [v, t, off]
        arr[i] = sdf_mesh(_ptr(v), v.shape[0], _ptr(t), t.shape[0], off.shape[0] - 1, _ptr(off))
    h = ctypes.c_void_p()
    ctx._check(lib.sdf_build_grids(ctx.handle, ctypes.addressof(arr), len(meshes), int(resolution),
                                   float(margin), ctypes.byref(h)), "sdf_build_grids")
    return Grids(ctx, h)


def sdf_grids_upload(ctx: Context, values, metas) -> Grids:
    """values: [L, n^3] (any float dtype, rounded to FP32); metas: rows of the
    oracle layout (origin[3], h, n, centre[3], radius, margin) or dicts."""
    vals = np.ascontiguousarray(np.asarray(values, dtype=np.float32).reshape(len(metas), -1))
    arr = (sdf_grid_meta * len(metas))()
    for i, m in enumerate(metas):
        if isinstance(m, dict):
            o, h, n, c, r, mg = m["origin"], m["h"], m["n"], m["center"], m["radius"], m["margin"]
        else:
            o, h, n, c, r, mg = m[0:3], m[3], m[4], m[5:8], m[8], m[9]
        arr[i].origin[:] = [float(x) for x in o]
        arr[i].h = float(h)
        arr[i].n = int(n)
        arr[i].center[:] = [float(x) for x in c]
        arr[i].radius = float(r)   # the library rounds it up by one ulp
        arr[i].margin = float(mg)
    h = ctypes.c_void_p()
    ctx._check(lib.sdf_grids_upload(ctx.handle, _ptr(vals), ctypes.addressof(arr), len(metas),
                                    ctypes.byref(h)), "sdf_grids_upload")
    return Grids(ctx, h)


class Robot:
    """Owns an sdf_robot (DH table + base + grids)."""

    def __init__(self, ctx: Context, dh, grids: Grids, base=None):
        dh = np.asarray(dh, dtype=np.float64).reshape(-1, 6)
        rows = (sdf_dh * max(len(dh), 1))()
        for j, r in enumerate(dh):
            rows[j] = sdf_dh(*[float(x) for x in r])
        b = None if base is None else np.ascontiguousarray(np.asarray(base, np.float32).reshape(12))
        h = ctypes.c_void_p()
        ctx._check(lib.sdf_robot_create(ctx.handle, ctypes.addressof(rows), len(dh), _ptr(b),
                                        grids.handle, ctypes.byref(h)), "sdf_robot_create")
        self.ctx, self.grids, self.handle, self.dof = ctx, grids, h, len(dh)
        self.n_links = self.dof + 1

    def close(self):
        if getattr(self, "handle", None):
            lib.sdf_robot_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sdf_forward_kinematics(ctx: Context, robot: Robot, q_dev, W: int, out_dev) -> None:
    ctx._check(lib.sdf_forward_kinematics(ctx.handle, robot.handle, _ptr(q_dev), int(W),
                                          _ptr(out_dev)), "sdf_forward_kinematics")


def check_trajectory(ctx: Context, robot: Robot, q_dev, W: int, points_dev, N: int, dist_dev,
                     argmin_link_dev, argmin_point_dev) -> None:
    """Enqueue the check on the context's stream (device buffers)."""
    ctx._check(lib.check_trajectory(ctx.handle, robot.handle, _ptr(q_dev), int(W), _ptr(points_dev),
                                    int(N), _ptr(dist_dev), _ptr(argmin_link_dev),
                                    _ptr(argmin_point_dev)), "check_trajectory")


def _requests(requests):
    arr = (sdf_check_request * max(len(requests), 1))()
    for i, r in enumerate(requests):
        robot, q, W, pts, N, d, al, ap = r[:8]
        mask = r[8] if len(r) > 8 else None
        arr[i] = sdf_check_request(robot.handle.value if hasattr(robot.handle, "value") else robot.handle,
                                   _ptr(q), int(W), _ptr(pts), int(N), _ptr(d), _ptr(al), _ptr(ap), _ptr(mask))
    return arr


def check_batch(ctx: Context, requests) -> None:
    """requests: sequence of (robot, q_dev, W, points_dev, N, dist_dev, link_dev, point_dev[, mask_dev])."""
    arr = _requests(requests)
    ctx._check(lib.check_batch(ctx.handle, ctypes.addressof(arr), len(requests)), "check_batch")


def sdf_autotune(ctx: Context, requests, repeats: int = 5):
    """Time the launch shapes on these requests; returns (waypoints per block,
    tile batch, median microseconds) of the fastest, which later calls reuse."""
    arr = _requests(requests)
    tw, tb, us = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    ctx._check(lib.sdf_autotune(ctx.handle, ctypes.addressof(arr), len(requests), int(repeats), ctypes.byref(tw),
                                ctypes.byref(tb), ctypes.byref(us)), "sdf_autotune")
    return int(tw.value), int(tb.value), float(us.value)


def sdf_measure_gather(ctx: Context, grids: "Grids"):
    """(random 4-byte gathers/s, random 8-corner cell reads/s) on these grids' values."""
    g, c = ctypes.c_double(), ctypes.c_double()
    ctx._check(lib.sdf_measure_gather(ctx.handle, grids.handle, ctypes.byref(g), ctypes.byref(c)),
               "sdf_measure_gather")
    return float(g.value), float(c.value)


def sdf_ctx_reserve(ctx: Context, max_points: int, max_waypoints: int, max_pairs: int,
                    max_requests: int) -> None:
    ctx._check(lib.sdf_ctx_reserve(ctx.handle, int(max_points), int(max_waypoints), int(max_pairs),
                                   int(max_requests)), "sdf_ctx_reserve")


def check_trajectory_host(ctx: Context, robot: Robot, q_host, W: int, points_host, N: int, dist_host,
                          argmin_link_host, argmin_point_host) -> int:
    """Host-buffer check (copies inside, synchronises); returns the status code
    (SDF_ERR_NONFINITE is returned, other errors raise)."""
    rc = lib.check_trajectory_host(ctx.handle, robot.handle, _ptr(q_host), int(W), _ptr(points_host),
                                   int(N), _ptr(dist_host), _ptr(argmin_link_host),
                                   _ptr(argmin_point_host))
    if rc not in (SDF_OK, SDF_ERR_NONFINITE):
        ctx._check(rc, "check_trajectory_host")
    return int(rc)


class HostCheck:
    """check_trajectory_host bound to fixed host buffers: the buffer addresses are
    taken once, and each call re-reads the buffers' current contents.  The object
    keeps the five arrays alive (so they cannot be freed or resized under it); a
    call costs one C call.  Returns the status code like check_trajectory_host."""

    def __init__(self, ctx: Context, robot: Robot, q_host, W: int, points_host, N: int, dist_host,
                 argmin_link_host, argmin_point_host):
        self._keep = (ctx, robot, q_host, points_host, dist_host, argmin_link_host, argmin_point_host)
        P, i32 = ctypes.c_void_p, ctypes.c_int32
        self._args = (ctx.handle, robot.handle, P(_ptr(q_host)), i32(int(W)), P(_ptr(points_host)),
                      i32(int(N)), P(_ptr(dist_host)), P(_ptr(argmin_link_host)), P(_ptr(argmin_point_host)))
        self._fn = lib.check_trajectory_host
        self._ctx = ctx

    def __call__(self) -> int:
        rc = self._fn(*self._args)
        if rc != SDF_OK and rc != SDF_ERR_NONFINITE:
            self._ctx._check(rc, "check_trajectory_host")
        return rc


def check_trajectory_noalloc(robot: Robot, stream, q_dev, W: int, points_dev, N: int, dist_dev,
                             argmin_link_dev, argmin_point_dev, status_dev=None) -> int:
    """The allocation-free check (no context, fixed-size device scratch); returns
    the status code of enqueueing (SDF_OK, SDF_ERR_INVALID_ARG or SDF_ERR_CUDA)."""
    return int(lib.check_trajectory_noalloc(robot.handle, _stream_handle(stream), _ptr(q_dev), int(W),
                                            _ptr(points_dev), int(N), _ptr(dist_dev), _ptr(argmin_link_dev),
                                            _ptr(argmin_point_dev), _ptr(status_dev)))


def sdf_debug_fail_alloc(k: int) -> None:
    """Make the k-th library allocation from now fail as out of memory (0 disarms)."""
    rc = int(lib.sdf_debug_fail_alloc(int(k)))
    if rc != SDF_OK:
        raise SdfError(rc, "sdf_debug_fail_alloc")


def sdf_debug_alloc_live():
    """(live allocations, their bytes, remaining fail countdown) of the library."""
    out = np.zeros(3, np.int64)
    lib.sdf_debug_alloc_live(_ptr(out[0:1]), _ptr(out[1:2]), _ptr(out[2:3]))
    return int(out[0]), int(out[1]), int(out[2])


class Server:
    """Serving engine (continuous batching of trajectory checks on one device)."""

    STAT_NAMES = ("p50_us", "p99_us", "mean_us", "completed", "rejected", "batches", "mean_batch",
                  "peak_in_flight", "pending", "max_us")

    def __init__(self, device: int = 0, memory_budget_bytes: int = 0, slots: int = 4, max_batch: int = 64,
                 max_waypoints: int = 16384, max_points: int = 100000, max_dof: int = 7,
                 batch_window_us: int = 0):
        cfg = sdf_server_config(int(device), int(memory_budget_bytes), int(slots), int(max_batch),
                                int(max_waypoints), int(max_points), int(max_dof), int(batch_window_us))
        h = ctypes.c_void_p()
        rc = lib.sdf_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != SDF_OK:
            raise SdfError(rc, "sdf_server_create failed")
        self.handle = h

    def set_cloud(self, points) -> int:
        p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
        return int(lib.sdf_server_set_cloud(self.handle, _ptr(p), int(p.shape[0])))

    def submit(self, robot: "Robot", q) -> int:
        """Queue a trajectory; returns its ticket (raises if rejected)."""
        qa = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, robot.dof)
        t = ctypes.c_uint64()
        rc = lib.sdf_server_submit(self.handle, robot.handle, _ptr(qa), int(qa.shape[0]), ctypes.byref(t))
        if rc != SDF_OK:
            raise SdfError(rc, "sdf_server_submit")
        self._w = getattr(self, "_w", {})
        self._w[int(t.value)] = int(qa.shape[0])
        return int(t.value)

    def poll(self, ticket: int, wait_us: int = -1):
        """(status, dist, link, point, latency_us); status SDF_PENDING while unfinished."""
        W = self._w[ticket]
        d = np.empty(W, np.float32)
        l = np.empty(W, np.int32)
        p = np.empty(W, np.int32)
        lat = ctypes.c_double()
        rc = int(lib.sdf_server_poll(self.handle, ctypes.c_uint64(ticket), int(wait_us), _ptr(d), _ptr(l), _ptr(p),
                                     ctypes.byref(lat)))
        if rc != SDF_PENDING and rc != SDF_ERR_TIMEOUT:
            self._w.pop(ticket, None)
        return rc, d, l, p, float(lat.value)

    def set_surrogate(self, surrogate, margin: float = 0.05, eps: float = 0.0):
        """Serve requests on the surrogate's grids in the surrogate form (None: grid form)."""
        rc = lib.sdf_server_set_surrogate(self.handle, surrogate.handle if surrogate is not None else None,
                                          float(margin), float(eps))
        if rc != SDF_OK:
            raise SdfError(rc, "sdf_server_set_surrogate")

    def stats(self, reset: bool = False) -> dict:
        out = np.zeros(10, dtype=np.float64)
        rc = lib.sdf_server_stats(self.handle, _ptr(out), 10, int(reset))
        if rc != SDF_OK:
            raise SdfError(rc, "sdf_server_stats")
        return dict(zip(self.STAT_NAMES, out.tolist()))

    def close(self):
        if getattr(self, "handle", None):
            lib.sdf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """Per-link MLP SDF surrogates (sdf_surrogate handle) on one context's device."""

    def __init__(self, ctx: Context, grids: "Grids", params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(grids.n_links, SDF_MLP_PARAMS)
        h = ctypes.c_void_p()
        ctx._check(lib.sdf_surrogate_create(ctx.handle, grids.handle, _ptr(p), ctypes.byref(h)),
                   "sdf_surrogate_create")
        self.ctx, self.grids, self.handle, self.n_links = ctx, grids, h, grids.n_links

    def params(self) -> np.ndarray:
        out = np.empty((self.n_links, SDF_MLP_PARAMS), dtype=np.float32)
        self.ctx._check(lib.sdf_surrogate_params(self.ctx.handle, self.handle, _ptr(out)), "sdf_surrogate_params")
        return out

    def grad(self, link: int, x, y, grad, loss=None):
        self.ctx._check(lib.sdf_surrogate_grad(self.ctx.handle, self.handle, int(link), _ptr(x), _ptr(y), _ptr(grad),
                                               _ptr(loss)), "sdf_surrogate_grad")

    def train(self, x, y, n: int, first_batch: int, steps: int, lr: float, loss=None):
        self.ctx._check(lib.sdf_surrogate_train(self.ctx.handle, self.handle, _ptr(x), _ptr(y), int(n),
                                                int(first_batch), int(steps), float(lr), _ptr(loss)),
                        "sdf_surrogate_train")

    def eval(self, link: int, x, n: int, f):
        self.ctx._check(lib.sdf_surrogate_eval(self.ctx.handle, self.handle, int(link), _ptr(x), int(n), _ptr(f)),
                        "sdf_surrogate_eval")

    def error(self, link: int, n: int, near_per_10: int = 0, band: float = 0.1, seed: int = 99):
        mx, mean = ctypes.c_float(), ctypes.c_float()
        self.ctx._check(lib.sdf_surrogate_error(self.ctx.handle, self.handle, int(link), int(n), int(near_per_10),
                                                float(band), ctypes.c_uint64(seed), ctypes.byref(mx),
                                                ctypes.byref(mean)), "sdf_surrogate_error")
        return float(mx.value), float(mean.value)

    def close(self):
        if getattr(self, "handle", None):
            lib.sdf_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sdf_surrogate_sample(ctx: Context, grids: "Grids", link: int, n: int, near_per_10: int, band: float, seed: int,
                         x, y, source=None):
    ctx._check(lib.sdf_surrogate_sample(ctx.handle, grids.handle, int(link), int(n), int(near_per_10), float(band),
                                        ctypes.c_uint64(seed), _ptr(x), _ptr(y), _ptr(source)),
               "sdf_surrogate_sample")


def check_trajectory_surrogate(ctx: Context, robot: "Robot", surrogate: Surrogate, q, W: int, points, N: int,
                               margin: float, eps: float, dist, link, point, rechecked=None, surrogate_dist=None):
    """The check with the surrogate in place of the grid lookup; waypoints below
    margin + eps are re-checked by the grid path (device buffers, asynchronous)."""
    ctx._check(lib.check_trajectory_surrogate(ctx.handle, robot.handle, surrogate.handle, _ptr(q), int(W), _ptr(points),
                                              int(N), float(margin), float(eps), _ptr(dist), _ptr(link), _ptr(point),
                                              _ptr(rechecked), _ptr(surrogate_dist)), "check_trajectory_surrogate")


def check_trajectory_robot_sdf(ctx: Context, robot: "Robot", origin, voxel: float, dims, reach: float, q, W: int,
                               points, N: int, dist, argmin_voxel) -> None:
    """The paper's Robot-SDF form of the check on an environment voxel grid
    (device buffers, asynchronous)."""
    env = sdf_env_grid((ctypes.c_float * 3)(*[float(x) for x in origin]), float(voxel),
                       (ctypes.c_int32 * 3)(*[int(x) for x in dims]), float(reach))
    ctx._check(lib.check_trajectory_robot_sdf(ctx.handle, robot.handle, ctypes.byref(env), _ptr(q), int(W),
                                              _ptr(points), int(N), _ptr(dist), _ptr(argmin_voxel)),
               "check_trajectory_robot_sdf")
