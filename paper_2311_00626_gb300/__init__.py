"""GB300-native projective TSDF integration (nvblox, arXiv 2311.00626).

Thin ctypes binding over the C ABI in ``include/tsdf.h`` (library
``libgb300tsdf.so``, built in-tree for sm_103a by ``build.py``).  The binding
only marshals arguments: torch CUDA tensors are passed as device pointers and
the current torch stream as the CUDA stream; every step of the integration
runs in the library's CUDA kernels.  There is no CPU fallback: loading fails
loudly if the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB, build as build_library

__all__ = ["TsdfError", "Pinhole", "Lidar", "MapOpts", "FrameDesc", "TsdfMap", "lib",
           "map_create", "map_create_ex", "integrate_depth", "integrate_lidar",
           "integrate_batch", "query_voxels", "map_sync", "map_num_blocks", "map_stats",
           "map_export", "map_reset", "map_destroy", "map_timing", "map_kernel_times",
           "MapBuffers", "integrate_depth_static", "STATIC_MAX_BLOCKS", "NUM_COUNTERS", "LAYER_TSDF",
           "LAYER_OCCUPANCY", "LAYER_COLOR", "STORAGE_FP32", "STORAGE_FP16", "STORAGE_FIXED16",
           "integrate_color", "query_color", "map_export_color", "map_decay_occupancy",
           "EsdfOpts", "map_import", "map_esdf_update", "map_esdf_export", "map_esdf_query",
           "map_esdf_stats", "map_walk_stats", "map_mesh", "integrate_batch_host", "frame_desc_host",
           "SENSOR_PINHOLE", "SENSOR_LIDAR", "EXPORTED_SYMBOLS", "LAUNCH_SPLIT", "LAUNCH_FUSED",
           "map_wait_test"]

STORAGE_FP32, STORAGE_FP16, STORAGE_FIXED16 = 0, 1, 2
LAYER_TSDF, LAYER_OCCUPANCY, LAYER_COLOR = 0, 1, 2
WEIGHT_CONSTANT, WEIGHT_INV_SQUARE, WEIGHT_DROPOFF = 0, 1, 2
STATIC_MAX_BLOCKS = 1 << 16  # TSDF_STATIC_MAX_BLOCKS
NUM_COUNTERS = 8  # TSDF_NUM_COUNTERS: u64 words of a caller-owned counters buffer
KEY_BITS, KEY_BIAS = 21, 1 << 20  # TSDF_KEY_BITS, TSDF_KEY_BIAS
SENSOR_PINHOLE, SENSOR_LIDAR = 0, 1
LAUNCH_SPLIT, LAUNCH_FUSED = 0, 1
_STATUS = {0: "TSDF_OK", -1: "TSDF_ERR_ARG", -2: "TSDF_ERR_CUDA", -3: "TSDF_ERR_CAPACITY",
           -4: "TSDF_ERR_TIMEOUT", -5: "TSDF_ERR_STATE"}
EXPORTED_SYMBOLS = ["map_create", "map_create_ex", "integrate_depth", "integrate_lidar",
                    "integrate_batch", "query_voxels", "map_sync", "map_num_blocks", "map_stats",
                    "map_export", "map_reset", "map_destroy", "map_timing", "map_kernel_times",
                    "integrate_depth_static", "integrate_color", "query_color",
                    "map_export_color", "map_decay_occupancy", "map_import", "map_esdf_update",
                    "map_esdf_export", "map_esdf_query", "map_esdf_stats", "map_walk_stats",
                    "map_mesh", "integrate_batch_host", "stage_frames", "map_wait_test"]


class TsdfError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_STATUS.get(code, code)}")
        self.code = code


class Pinhole(ctypes.Structure):
    _fields_ = [("fu", ctypes.c_float), ("fv", ctypes.c_float), ("cu", ctypes.c_float),
                ("cv", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Lidar(ctypes.Structure):
    _fields_ = [("n_az", ctypes.c_int32), ("n_el", ctypes.c_int32),
                ("theta_start", ctypes.c_float), ("phi_start", ctypes.c_float),
                ("el_fov", ctypes.c_float), ("min_range", ctypes.c_float),
                ("max_range", ctypes.c_float)]


class MapOpts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("max_blocks", ctypes.c_int64),
                ("hash_capacity", ctypes.c_int64), ("lidar_nearest", ctypes.c_int32),
                ("lidar_guard", ctypes.c_float), ("alloc_tile_h", ctypes.c_int32),
                ("integrate_ctas_per_sm", ctypes.c_int32), ("layer", ctypes.c_int32),
                ("l_occ", ctypes.c_float), ("l_free", ctypes.c_float),
                ("weighting", ctypes.c_int32), ("dropoff", ctypes.c_float),
                ("launch_mode", ctypes.c_int32)]


class FrameDesc(ctypes.Structure):
    _fields_ = [("map", ctypes.c_int32), ("kind", ctypes.c_int32), ("pinhole", Pinhole),
                ("lidar", Lidar), ("depth_dev", ctypes.c_void_p),
                ("T_world_sensor", ctypes.c_double * 16), ("color_dev", ctypes.c_void_p)]


class EsdfOpts(ctypes.Structure):
    _fields_ = [("site_eps", ctypes.c_float), ("min_weight", ctypes.c_float),
                ("max_dist_vox", ctypes.c_int32)]


class MapBuffers(ctypes.Structure):
    """Caller-owned FP32 map storage for integrate_depth_static (see tsdf.h)."""
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("pool", ctypes.c_void_p), ("block_keys", ctypes.c_void_p),
                ("counters", ctypes.c_void_p), ("hash_capacity", ctypes.c_int64),
                ("max_blocks", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if stale) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_library()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing")
            L = ctypes.CDLL(path)
            P, I, L64, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
            PP = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "map_create": ([F, I, F, PP], I),
                "map_create_ex": ([F, I, F, ctypes.POINTER(MapOpts), PP], I),
                "integrate_depth": ([P, P, ctypes.POINTER(Pinhole), P, P], I),
                "integrate_lidar": ([P, P, ctypes.POINTER(Lidar), P, P], I),
                "integrate_batch": ([P, I, ctypes.POINTER(FrameDesc), I, P], I),
                "integrate_batch_host": ([P, I, ctypes.POINTER(FrameDesc), I, P, L64, P], I),
                "stage_frames": ([P, P, P, I, P], I),
                "query_voxels": ([P, P, L64, P, P, P], I),
                "map_sync": ([P], I),
                "map_num_blocks": ([P, ctypes.POINTER(ctypes.c_int64)], I),
                "map_stats": ([P, P], I),
                "map_export": ([P, P, P, P, L64], I),
                "map_reset": ([P, P], I),
                "map_destroy": ([P], I),
                "map_timing": ([P, I], I),
                "map_walk_stats": ([P, I], I),
                "map_wait_test": ([P, I], I),
                "map_mesh": ([P, F, I, P, P, P, L64, ctypes.POINTER(ctypes.c_int64), P], I),
                "map_kernel_times": ([P, P, ctypes.POINTER(ctypes.c_int64)], I),
                "integrate_depth_static": ([ctypes.POINTER(MapBuffers), F, I, F, P,
                                            ctypes.POINTER(Pinhole), P, P], I),
                "integrate_color": ([P, P, P, ctypes.POINTER(Pinhole), P, P], I),
                "query_color": ([P, P, L64, P, P, P], I),
                "map_export_color": ([P, P, P, P, L64], I),
                "map_decay_occupancy": ([P, F, F, P], I),
                "map_import": ([P, P, P, P, L64], I),
                "map_esdf_update": ([P, ctypes.POINTER(EsdfOpts), P], I),
                "map_esdf_export": ([P, P, P, L64], I),
                "map_esdf_query": ([P, P, L64, P, P], I),
                "map_esdf_stats": ([P, P], I),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(code: int, what: str):
    if code != 0:
        raise TsdfError(code, what)


def _pose(T) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return (ctypes.c_double * 16)(*a.tolist())


def _pose_arg(T):
    """A pose as a call argument: the array's own memory when it already is
    16 contiguous doubles (the caller holds it for the call), else a copy."""
    if type(T) is np.ndarray and T.dtype == np.float64 and T.size == 16 and T.flags.c_contiguous:
        return T.ctypes.data
    return _pose(T)


_torch = None
_raw_stream = None


def _stream(stream) -> int | None:
    """The CUDA stream handle of `stream`, or of torch's current stream."""
    global _torch, _raw_stream
    if stream is None:
        if _torch is None:
            import torch
            torch.cuda.init()  # the raw getter below does not initialise CUDA itself
            _torch = torch
            # the raw getter avoids building a Stream object on every call
            _raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if _raw_stream is not None:
            return _raw_stream(_torch._C._cuda_getDevice())
        return _torch.cuda.current_stream().cuda_stream
    return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream


def _dptr(t) -> int:
    """Device pointer of a contiguous float32 CUDA tensor (or a raw int)."""
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def pinhole(sensor: dict) -> Pinhole:
    return Pinhole(sensor["fu"], sensor["fv"], sensor["cu"], sensor["cv"], sensor["width"],
                   sensor["height"])


def lidar(sensor: dict) -> Lidar:
    return Lidar(sensor["n_az"], sensor["n_el"], sensor["theta_start"], sensor["phi_start"],
                 sensor["el_fov"], sensor["min_range"], sensor["max_range"])


# ---- the C ABI under its own names -----------------------------------------------

def map_create(voxel_size: float, truncation_voxels: int, max_weight: float) -> int:
    h = ctypes.c_void_p()
    _check(lib().map_create(voxel_size, truncation_voxels, max_weight, ctypes.byref(h)),
           "map_create")
    return h.value


def map_create_ex(voxel_size, truncation_voxels, max_weight, storage=STORAGE_FP32, max_blocks=0,
                  hash_capacity=0, lidar_nearest=False, lidar_guard=0.0, alloc_tile_h=0,
                  integrate_ctas_per_sm=0, layer=LAYER_TSDF, l_occ=0.0, l_free=0.0,
                  weighting=WEIGHT_CONSTANT, dropoff=0.0, launch_mode=LAUNCH_SPLIT) -> int:
    h = ctypes.c_void_p()
    o = MapOpts(storage, max_blocks, hash_capacity, int(lidar_nearest), lidar_guard, alloc_tile_h,
                integrate_ctas_per_sm, layer, l_occ, l_free, weighting, dropoff, launch_mode)
    _check(lib().map_create_ex(voxel_size, truncation_voxels, max_weight, ctypes.byref(o),
                               ctypes.byref(h)), "map_create_ex")
    return h.value


def integrate_depth(m: int, depth, intr: Pinhole, T_world_cam, stream=None):
    _check(lib().integrate_depth(m, _dptr(depth), ctypes.byref(intr), _pose_arg(T_world_cam),
                                 _stream(stream)), "integrate_depth")


def integrate_lidar(m: int, rng, intr: Lidar, T_world_lidar, stream=None):
    _check(lib().integrate_lidar(m, _dptr(rng), ctypes.byref(intr), _pose_arg(T_world_lidar),
                                 _stream(stream)), "integrate_lidar")


def integrate_color(m: int, depth, rgba, intr: Pinhole, T_world_cam, stream=None):
    """depth: float32 [H, W] device tensor; rgba: uint32 (int32) [H, W] device
    tensor, r in the low byte."""
    _check(lib().integrate_color(m, _dptr(depth), _dptr(rgba), ctypes.byref(intr),
                                 _pose_arg(T_world_cam), _stream(stream)), "integrate_color")


def integrate_batch(maps, frames, stream=None):
    """maps: sequence of map handles; frames: sequence of FrameDesc."""
    arr_m = (ctypes.c_void_p * len(maps))(*maps)
    arr_f = (FrameDesc * len(frames))(*frames)
    _check(lib().integrate_batch(arr_m, len(maps), arr_f, len(frames), _stream(stream)),
           "integrate_batch")


def integrate_batch_host(maps, frames, staging, stream=None):
    """frames: FrameDesc with host image pointers (frame_desc_host);
    staging: a CUDA uint8 (or any) tensor of at least two sub-batches' image
    bytes, 256-byte aligned."""
    arr_m = (ctypes.c_void_p * len(maps))(*maps)
    arr_f = (FrameDesc * len(frames))(*frames)
    nbytes = staging.numel() * staging.element_size()
    _check(lib().integrate_batch_host(arr_m, len(maps), arr_f, len(frames), staging.data_ptr(), nbytes,
                                      _stream(stream)), "integrate_batch_host")


def stage_frames(src_host, dst_dev, nbytes, stream=None):
    """Enqueue host-to-device copies src_host[i] -> dst_dev[i] of nbytes[i]
    bytes (pointers as ints) on `stream` in one C call."""
    n = len(src_host)
    if not (len(dst_dev) == len(nbytes) == n):
        raise ValueError("stage_frames: arrays of different lengths")
    src = (ctypes.c_void_p * n)(*src_host)
    dst = (ctypes.c_void_p * n)(*dst_dev)
    cnt = (ctypes.c_int64 * n)(*nbytes)
    _check(lib().stage_frames(src, dst, cnt, n, _stream(stream)), "stage_frames")


def query_voxels(m: int, pts, dist, weight, stream=None):
    n = pts.shape[0] if hasattr(pts, "shape") else 0
    _check(lib().query_voxels(m, _dptr(pts), n, _dptr(dist), _dptr(weight), _stream(stream)),
           "query_voxels")


def query_color(m: int, pts, rgb, weight, stream=None):
    n = pts.shape[0] if hasattr(pts, "shape") else 0
    _check(lib().query_color(m, _dptr(pts), n, _dptr(rgb), _dptr(weight), _stream(stream)),
           "query_color")


def map_sync(m: int) -> int:
    return lib().map_sync(m)


def map_num_blocks(m: int) -> int:
    out = ctypes.c_int64()
    _check(lib().map_num_blocks(m, ctypes.byref(out)), "map_num_blocks")
    return out.value


def map_stats(m: int) -> dict:
    out = np.zeros(9, np.int64)
    _check(lib().map_stats(m, out.ctypes.data_as(ctypes.c_void_p)), "map_stats")
    return {"blocks": int(out[0]), "voxel_updates": int(out[1]), "frames": int(out[2]),
            "status_bits": int(out[3]), "block_visits": int(out[4]), "launches": int(out[5]),
            "segments": int(out[6]), "cells": int(out[7]), "block_frame_pairs": int(out[8])}


def map_walk_stats(m: int, enable: bool = True):
    """Count band segments and walked cells (map_stats "segments", "cells")."""
    _check(lib().map_walk_stats(m, int(enable)), "map_walk_stats")


def map_wait_test(m: int, extra_ctas: int):
    """Test hook: fused launches wait for extra_ctas CTAs that do not exist
    (their bounded wait runs out: TSDF_ERR_TIMEOUT); 0 restores them."""
    _check(lib().map_wait_test(m, int(extra_ctas)), "map_wait_test")


def map_timing(m: int, enable: bool = True):
    _check(lib().map_timing(m, int(enable)), "map_timing")


def map_kernel_times(m: int):
    """(alloc_ms, integrate_ms, calls) summed over the recorded calls."""
    out = np.zeros(2, np.float64)
    calls = ctypes.c_int64()
    _check(lib().map_kernel_times(m, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(calls)),
           "map_kernel_times")
    return float(out[0]), float(out[1]), int(calls.value)


def map_export(m: int, with_values: bool = True):
    """(keys int32[n,3] sorted by (x,y,z), D float32[n,512], W float32[n,512])."""
    n = map_num_blocks(m)
    keys = np.zeros((n, 3), np.int32)
    D = np.zeros((n, 512), np.float32) if with_values else None
    W = np.zeros((n, 512), np.float32) if with_values else None
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None  # noqa: E731
    _check(lib().map_export(m, vp(keys), vp(D), vp(W), n), "map_export")
    return keys, D, W


def map_export_color(m: int):
    """(keys int32[n,3] sorted by (x,y,z), rgb float32[n,512,3], W float32[n,512])."""
    n = map_num_blocks(m)
    keys = np.zeros((n, 3), np.int32)
    rgb = np.zeros((n, 512, 3), np.float32)
    W = np.zeros((n, 512), np.float32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().map_export_color(m, vp(keys), vp(rgb), vp(W), n), "map_export_color")
    return keys, rgb, W


def map_decay_occupancy(m: int, decay_occ: float, decay_free: float, stream=None):
    _check(lib().map_decay_occupancy(m, decay_occ, decay_free, _stream(stream)),
           "map_decay_occupancy")


def map_import(m: int, keys, D, W=None):
    """Write blocks (keys int32 [n,3], D / W float32 [n,512]) into the map."""
    keys = np.ascontiguousarray(keys, np.int32)
    D = np.ascontiguousarray(D, np.float32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None  # noqa: E731
    W = None if W is None else np.ascontiguousarray(W, np.float32)
    _check(lib().map_import(m, vp(keys), vp(D), vp(W), len(keys)), "map_import")


def map_esdf_update(m: int, site_eps: float | None = None, min_weight: float = 1e-4,
                    max_dist_vox: int = 64, stream=None):
    o = None
    if site_eps is not None:
        o = ctypes.byref(EsdfOpts(site_eps, min_weight, max_dist_vox))
    _check(lib().map_esdf_update(m, o, _stream(stream)), "map_esdf_update")


def map_esdf_export(m: int):
    """(keys int32 [n,3] sorted by (x,y,z), states uint32 [n,512])."""
    n = map_num_blocks(m)
    keys = np.zeros((n, 3), np.int32)
    st = np.zeros((n, 512), np.uint32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().map_esdf_export(m, vp(keys), vp(st), n), "map_esdf_export")
    return keys, st


def map_esdf_query(m: int, pts, dist, stream=None):
    n = pts.shape[0] if hasattr(pts, "shape") else 0
    _check(lib().map_esdf_query(m, _dptr(pts), n, _dptr(dist), _stream(stream)), "map_esdf_query")


def map_esdf_stats(m: int) -> dict:
    out = np.zeros(4, np.int64)
    _check(lib().map_esdf_stats(m, out.ctypes.data_as(ctypes.c_void_p)), "map_esdf_stats")
    return dict(zip(["iterations", "swept", "pulled", "cleared"], (int(x) for x in out)))


def map_mesh(m: int, min_weight: float = 1e-4, changed_only: bool = False, with_keys: bool = True,
             cap: int = 0, stream=None):
    """Marching-cubes triangles: (pos float32 [t,3,3], keys int32 [t,3,4] or
    None, cube int32 [t,3] or None) as CUDA tensors.  When cap is too small
    a full extraction is retried with room for all triangles; a changed_only
    extraction raises (its changed blocks were consumed)."""
    import torch
    cap = cap or (1 << 20)
    n = ctypes.c_int64()
    while True:
        pos = torch.empty((cap, 3, 3), dtype=torch.float32, device="cuda")
        keys = torch.empty((cap, 3, 4), dtype=torch.int32, device="cuda") if with_keys else None
        cube = torch.empty((cap, 3), dtype=torch.int32, device="cuda") if with_keys else None
        code = lib().map_mesh(m, min_weight, int(changed_only), _dptr(pos),
                              _dptr(keys) if keys is not None else None,
                              _dptr(cube) if cube is not None else None, cap, ctypes.byref(n),
                              _stream(stream))
        if code == -3 and not changed_only:  # TSDF_ERR_CAPACITY: retry with room for all
            cap = int(n.value)
            continue
        _check(code, "map_mesh")
        t = int(n.value)
        return pos[:t], (keys[:t] if keys is not None else None), (cube[:t] if cube is not None else None)


def map_reset(m: int, stream=None):
    _check(lib().map_reset(m, _stream(stream)), "map_reset")


def map_destroy(m: int):
    _check(lib().map_destroy(m), "map_destroy")


def integrate_depth_static(buffers: MapBuffers, voxel_size: float, truncation_voxels: int,
                           max_weight: float, depth, intr: Pinhole, T_world_cam, stream=None):
    """Allocation-free integration of one pinhole frame into caller-owned
    storage; raises TsdfError with the C status on failure."""
    _check(lib().integrate_depth_static(ctypes.byref(buffers), voxel_size, truncation_voxels,
                                        max_weight, _dptr(depth), ctypes.byref(intr),
                                        _pose_arg(T_world_cam), _stream(stream)),
           "integrate_depth_static")


class TsdfMap:
    """Owning wrapper around a map handle."""

    def __init__(self, voxel_size: float, truncation_voxels: int = 4, max_weight: float = 100.0,
                 storage: int = STORAGE_FP32, max_blocks: int = 0, hash_capacity: int = 0,
                 lidar_nearest: bool = False, lidar_guard: float = 0.0, alloc_tile_h: int = 0,
                 integrate_ctas_per_sm: int = 0, layer: int = LAYER_TSDF, l_occ: float = 0.0,
                 l_free: float = 0.0, weighting: int = WEIGHT_CONSTANT, dropoff: float = 0.0,
                 launch_mode: int = LAUNCH_SPLIT):
        self.handle = map_create_ex(voxel_size, truncation_voxels, max_weight, storage,
                                    max_blocks, hash_capacity, lidar_nearest, lidar_guard,
                                    alloc_tile_h, integrate_ctas_per_sm, layer, l_occ, l_free,
                                    weighting, dropoff, launch_mode)
        self.voxel_size = voxel_size
        self.storage = storage

    def integrate(self, sensor: dict, T, depth, stream=None):
        if sensor["kind"] == "pinhole":
            integrate_depth(self.handle, depth, pinhole(sensor), T, stream)
        else:
            integrate_lidar(self.handle, depth, lidar(sensor), T, stream)

    def integrate_color(self, sensor: dict, T, depth, rgba, stream=None):
        integrate_color(self.handle, depth, rgba, pinhole(sensor), T, stream)

    def frame_desc(self, index: int, sensor: dict, T, depth, rgba=None) -> FrameDesc:
        return frame_desc(index, sensor, T, depth, rgba)

    def sync(self) -> int:
        return map_sync(self.handle)

    def num_blocks(self) -> int:
        return map_num_blocks(self.handle)

    def stats(self) -> dict:
        return map_stats(self.handle)

    def export(self, with_values: bool = True):
        return map_export(self.handle, with_values)

    def export_color(self):
        return map_export_color(self.handle)

    def query(self, pts, dist, weight, stream=None):
        query_voxels(self.handle, pts, dist, weight, stream)

    def query_color(self, pts, rgb, weight, stream=None):
        query_color(self.handle, pts, rgb, weight, stream)

    def import_blocks(self, keys, D, W=None):
        map_import(self.handle, keys, D, W)

    def esdf_update(self, site_eps: float | None = None, min_weight: float = 1e-4,
                    max_dist_vox: int = 64, stream=None):
        map_esdf_update(self.handle, site_eps, min_weight, max_dist_vox, stream)

    def esdf_export(self):
        return map_esdf_export(self.handle)

    def esdf_query(self, pts, dist, stream=None):
        map_esdf_query(self.handle, pts, dist, stream)

    def mesh(self, min_weight: float = 1e-4, changed_only: bool = False, with_keys: bool = True,
             cap: int = 0, stream=None):
        return map_mesh(self.handle, min_weight, changed_only, with_keys, cap, stream)

    def esdf_stats(self) -> dict:
        return map_esdf_stats(self.handle)

    def decay(self, decay_occ: float, decay_free: float, stream=None):
        map_decay_occupancy(self.handle, decay_occ, decay_free, stream)

    def reset(self, stream=None):
        map_reset(self.handle, stream)

    def close(self):
        if self.handle:
            map_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def frame_desc_host(map_index: int, sensor: dict, T, depth, rgba=None) -> FrameDesc:
    """As frame_desc with host images (contiguous CPU tensors, pinned for
    overlapped copies) for integrate_batch_host."""
    for t in (depth, rgba):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError("expected a contiguous host tensor")
    fd = frame_desc(map_index, sensor, T, depth.data_ptr())
    fd.color_dev = rgba.data_ptr() if rgba is not None else None
    return fd


def frame_desc(map_index: int, sensor: dict, T, depth, rgba=None) -> FrameDesc:
    fd = FrameDesc()
    fd.map = map_index
    if sensor["kind"] == "pinhole":
        fd.kind = SENSOR_PINHOLE
        fd.pinhole = pinhole(sensor)
    else:
        fd.kind = SENSOR_LIDAR
        fd.lidar = lidar(sensor)
    fd.depth_dev = _dptr(depth)
    if type(T) is np.ndarray and T.dtype == np.float64 and T.size == 16 and T.flags.c_contiguous:
        ctypes.memmove(ctypes.addressof(fd) + FrameDesc.T_world_sensor.offset, T.ctypes.data, 128)
    else:
        fd.T_world_sensor = _pose(T)
    fd.color_dev = _dptr(rgba) if rgba is not None else None
    return fd
