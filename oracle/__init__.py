"""CPU oracle for projective TSDF integration — TEST INFRASTRUCTURE ONLY.

A plain FP64 restatement of nvblox's frame integration (Sec. IV-B, Eq. 1-3)
in ``tsdf_oracle.cpp``, of its incremental ESDF (Sec. IV-C) in
``esdf_oracle.cpp`` and of marching-cubes meshing in ``mesh_oracle.cpp``,
loaded through ctypes.  Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import this
module; the product path never does, and it shares no code with the CUDA
path.  See the header of ``tsdf_oracle.cpp`` for the precision contract
(FP64 values, prescribed FP32 decisions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("tsdf_oracle.cpp", "esdf_oracle.cpp", "mesh_oracle.cpp")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle sources into liboracle.so (g++, FP contraction off)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(p) for p in _SRCS)):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           *_SRCS, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(cmd, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, F, I, L, D = (ctypes.c_void_p, ctypes.c_float, ctypes.c_int32, ctypes.c_int64,
                             ctypes.c_double)
            lib.orc_create.argtypes = [F, I, F]
            lib.orc_create.restype = P
            lib.orc_destroy.argtypes = [P]
            lib.orc_set_lidar_sampling.argtypes = [P, I, F]
            lib.orc_set_occupancy.argtypes = [P, F, F]
            lib.orc_set_weighting.argtypes = [P, I, F]
            lib.orc_decay_occupancy.argtypes = [P, F, F]
            lib.orc_decay_occupancy.restype = I
            lib.orc_integrate_pinhole.argtypes = [P, P, I, I, F, F, F, F, P]
            lib.orc_integrate_pinhole.restype = I
            lib.orc_integrate_color.argtypes = [P, P, P, I, I, F, F, F, F, P]
            lib.orc_integrate_color.restype = I
            lib.orc_export_color.argtypes = [P, P, L]
            lib.orc_export_color.restype = L
            lib.orc_integrate_lidar.argtypes = [P, P, I, I, F, F, F, F, F, P]
            lib.orc_integrate_lidar.restype = I
            lib.orc_num_blocks.argtypes = [P]
            lib.orc_num_blocks.restype = L
            lib.orc_export.argtypes = [P, P, P, P, L]
            lib.orc_export.restype = L
            lib.orc_last_band.argtypes = [P, P, L]
            lib.orc_last_band.restype = L
            lib.orc_counters.argtypes = [P, P]
            lib.orc_atan2_dec.argtypes = [F, F]
            lib.orc_atan2_dec.restype = F
            lib.orc_dda.argtypes = [P, P, F, F, P]
            lib.orc_dda.restype = I
            lib.esdf_orc_create.argtypes = [F, F, F, I]
            lib.esdf_orc_create.restype = P
            lib.esdf_orc_destroy.argtypes = [P]
            lib.esdf_orc_set_occupancy.argtypes = [P]
            lib.esdf_orc_update.argtypes = [P, P, P, P, L, P]
            lib.esdf_orc_update.restype = L
            lib.esdf_orc_num_blocks.argtypes = [P]
            lib.esdf_orc_num_blocks.restype = L
            lib.esdf_orc_export.argtypes = [P, P, P, L]
            lib.esdf_orc_export.restype = L
            lib.esdf_orc_counters.argtypes = [P, P]
            lib.mesh_orc_extract.argtypes = [P, P, P, L, P, F, F, P, P, P, L]
            lib.mesh_orc_extract.restype = L
            lib.mesh_orc_case.argtypes = [I, P]
            lib.mesh_orc_case.restype = I
            _lib = lib
            del D
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleMap:
    """One TSDF layer held by the oracle (map_create analogue)."""

    def __init__(self, voxel_size: float, truncation_voxels: int = 4, max_weight: float = 100.0):
        self._lib = _load()
        self._h = self._lib.orc_create(voxel_size, truncation_voxels, max_weight)
        self.voxel_size = float(np.float32(voxel_size))
        self.truncation_voxels = truncation_voxels
        self.max_weight = max_weight

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_lidar_sampling(self, nearest: bool = False, guard: float = 0.0):
        self._lib.orc_set_lidar_sampling(self._h, int(nearest), guard)

    def set_weighting(self, mode: int, dropoff: float = 0.0):
        """TSDF weight f_w: 0 constant, 1 inverse square depth, 2 constant with
        drop-off behind the surface, 3 both."""
        self._lib.orc_set_weighting(self._h, mode, dropoff)

    def set_occupancy(self, l_occ: float, l_free: float):
        """Occupancy layer: D becomes the log-odds, W the number of updates."""
        self._lib.orc_set_occupancy(self._h, l_occ, l_free)

    def decay_occupancy(self, decay_occ: float, decay_free: float):
        """One decay step: occupied log-odds drop by decay_occ, free ones rise
        by decay_free, neither crossing 0."""
        if self._lib.orc_decay_occupancy(self._h, decay_occ, decay_free) != 0:
            raise RuntimeError("oracle decay_occupancy failed")

    def integrate(self, sensor: dict, T: np.ndarray, depth: np.ndarray):
        depth = np.ascontiguousarray(depth, np.float32)
        T = np.ascontiguousarray(T, np.float64).reshape(16)
        if sensor["kind"] == "pinhole":
            assert depth.shape == (sensor["height"], sensor["width"])
            rc = self._lib.orc_integrate_pinhole(self._h, _p(depth), sensor["width"],
                                                 sensor["height"], sensor["fu"], sensor["fv"],
                                                 sensor["cu"], sensor["cv"], _p(T))
        else:
            assert depth.shape == (sensor["n_el"], sensor["n_az"])
            rc = self._lib.orc_integrate_lidar(self._h, _p(depth), sensor["n_az"], sensor["n_el"],
                                               sensor["theta_start"], sensor["phi_start"],
                                               sensor["el_fov"], sensor["min_range"],
                                               sensor["max_range"], _p(T))
        if rc != 0:
            raise RuntimeError(f"oracle integrate failed ({rc})")

    def integrate_color(self, sensor: dict, T: np.ndarray, depth: np.ndarray, rgba: np.ndarray):
        """Colour layer: a registered depth image and uint32 RGBA image (r in
        the low byte); voxels within tau of the surface average their pixel's
        colour."""
        depth = np.ascontiguousarray(depth, np.float32)
        rgba = np.ascontiguousarray(rgba, np.uint32)
        T = np.ascontiguousarray(T, np.float64).reshape(16)
        assert depth.shape == rgba.shape == (sensor["height"], sensor["width"])
        rc = self._lib.orc_integrate_color(self._h, _p(depth), _p(rgba), sensor["width"],
                                           sensor["height"], sensor["fu"], sensor["fv"],
                                           sensor["cu"], sensor["cv"], _p(T))
        if rc != 0:
            raise RuntimeError(f"oracle integrate_color failed ({rc})")

    def export_color(self) -> np.ndarray:
        """float64 [n, 512, 3] colours, blocks in export order."""
        n = self.num_blocks()
        rgb = np.zeros((n, 512, 3), np.float64)
        assert self._lib.orc_export_color(self._h, _p(rgb), n) == n
        return rgb

    def num_blocks(self) -> int:
        return int(self._lib.orc_num_blocks(self._h))

    def export(self, with_values: bool = True):
        """(keys int32[n,3] sorted by (x,y,z), D float64[n,512], W float64[n,512])."""
        n = self.num_blocks()
        keys = np.zeros((n, 3), np.int32)
        D = np.zeros((n, 512), np.float64) if with_values else None
        W = np.zeros((n, 512), np.float64) if with_values else None
        got = self._lib.orc_export(self._h, _p(keys), _p(D) if with_values else None,
                                   _p(W) if with_values else None, n)
        assert got == n
        return keys, D, W

    def last_band(self) -> np.ndarray:
        n = int(self.counters()["band_blocks"])
        keys = np.zeros((n, 3), np.int32)
        got = self._lib.orc_last_band(self._h, _p(keys), n)
        assert got == n
        return keys

    def counters(self) -> dict:
        out = np.zeros(6, np.int64)
        self._lib.orc_counters(self._h, _p(out))
        names = ["candidates", "band_blocks", "new_blocks", "voxels_updated", "truncated_rays",
                 "total_updates"]
        return dict(zip(names, (int(x) for x in out)))


def atan2_dec(y: float, x: float) -> float:
    return float(_load().orc_atan2_dec(y, x))


def dda(o, direction, s0: float, s1: float) -> np.ndarray:
    """Cells (anchor-relative, int32[n,3]) of the oracle's block traversal."""
    o = np.ascontiguousarray(o, np.float32)
    direction = np.ascontiguousarray(direction, np.float32)
    cells = np.zeros((32, 3), np.int32)
    n = _load().orc_dda(_p(o), _p(direction), s0, s1, _p(cells))
    return cells[:n].copy()


# ESDF state word (see esdf_oracle.cpp): 9-bit parent offsets, then flags
ESDF_OBS, ESDF_SITE, ESDF_PAR, ESDF_INSIDE = 1 << 27, 1 << 28, 1 << 29, 1 << 30


def esdf_offsets(states: np.ndarray) -> np.ndarray:
    """int32 [..., 3] parent offsets of ESDF state words."""
    s = states.astype(np.int64)
    raw = np.stack([(s >> (9 * a)) & 511 for a in range(3)], -1)
    return np.where(raw >= 256, raw - 512, raw).astype(np.int32)


class EsdfOracle:
    """Incremental ESDF over TSDF blocks (Sec. IV-C), integer parent offsets."""

    def __init__(self, voxel_size: float, site_eps: float, min_weight: float, max_dist_vox: int,
                 occupancy: bool = False):
        """occupancy: D holds log-odds and sites follow the occupancy rule
        (occupied voxels next to free ones)."""
        self._lib = _load()
        self._h = self._lib.esdf_orc_create(voxel_size, site_eps, min_weight, max_dist_vox)
        if not self._h:
            raise ValueError("bad ESDF parameters")
        if occupancy:
            self._lib.esdf_orc_set_occupancy(self._h)

    def close(self):
        if self._h:
            self._lib.esdf_orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, keys: np.ndarray, D: np.ndarray, W: np.ndarray, changed=None) -> int:
        """keys int32 [n,3], D / W float32 [n,512] (the TSDF blocks), changed
        bool [n] (default: all).  Returns the lowering iterations."""
        keys = np.ascontiguousarray(keys, np.int32)
        D = np.ascontiguousarray(D, np.float32)
        W = np.ascontiguousarray(W, np.float32)
        n = len(keys)
        ch = np.ones(n, np.uint8) if changed is None else np.ascontiguousarray(changed, np.uint8)
        return int(self._lib.esdf_orc_update(self._h, _p(keys), _p(D), _p(W), n, _p(ch)))

    def export(self):
        """(keys int32 [n,3] sorted by (x,y,z), states uint32 [n,512])."""
        n = int(self._lib.esdf_orc_num_blocks(self._h))
        keys = np.zeros((n, 3), np.int32)
        st = np.zeros((n, 512), np.uint32)
        assert self._lib.esdf_orc_export(self._h, _p(keys), _p(st), n) == n
        return keys, st

    def counters(self) -> dict:
        out = np.zeros(4, np.int64)
        self._lib.esdf_orc_counters(self._h, _p(out))
        return dict(zip(["iterations", "swept", "pulled", "cleared"], (int(x) for x in out)))


def mesh_extract(keys, D, W, voxel_size: float, min_weight: float = 1e-4, blocks=None):
    """Marching-cubes triangles of the cubes of `blocks` (bool [n], default
    all): (cube int32 [t,3] = voxel index of its corner 0, vertex keys int32
    [t,3,4] = lower-corner voxel index and edge axis, positions float64
    [t,3,3] in metres)."""
    keys = np.ascontiguousarray(keys, np.int32)
    D = np.ascontiguousarray(D, np.float32)
    W = np.ascontiguousarray(W, np.float32)
    n = len(keys)
    sel = np.ones(n, np.uint8) if blocks is None else np.ascontiguousarray(blocks, np.uint8)
    lib = _load()
    cap = 1 << 16
    while True:
        cube = np.zeros((cap, 3), np.int32)
        k = np.zeros((cap, 3, 4), np.int32)
        pos = np.zeros((cap, 3, 3), np.float64)
        t = int(lib.mesh_orc_extract(_p(keys), _p(D), _p(W), n, _p(sel), voxel_size, min_weight,
                                     _p(cube), _p(k), _p(pos), cap))
        if t <= cap:
            return cube[:t], k[:t], pos[:t]
        cap = t


def mesh_case(inside_mask: int) -> np.ndarray:
    """Triangles (edge numbers, int32 [t,3]) of one cube configuration."""
    e = np.zeros(36, np.int32)
    t = int(_load().mesh_orc_case(inside_mask, _p(e)))
    return e[:3 * t].reshape(t, 3)
