"""Seeded synthetic inputs for the TSDF integration path (inputs only).

Scenes, trajectories and depth / range images are produced by ``synth.c``
(exact FP64 ray casting, counter-based noise).  Nothing here performs any step
of the integration method; the oracle tests and the CUDA path's tests and
benchmark both draw their inputs from this module.

The workload recipes mirror the shapes of the paper's evaluation (Sec. V:
indoor RGB-D rooms, a 64-beam spinning LiDAR) with seeded stand-ins for the
datasets, which are not available here.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

NPAR = 9
ROOM, BOX, SPHERE, CYL, PLANE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            P = ctypes.c_void_p
            I = ctypes.c_int32
            U = ctypes.c_uint64
            lib.synth_render_pinhole.argtypes = [P, I, P, D, D, D, D, I, I, D, D, D, U, U, P]
            lib.synth_render_pinhole.restype = None
            lib.synth_render_lidar.argtypes = [P, I, P, I, I, D, D, D, D, D, D, U, U, P]
            lib.synth_render_lidar.restype = None
            lib.synth_room_scene.argtypes = [U, D, D, D, I, I, D, D, D, D, P]
            lib.synth_room_scene.restype = I
            lib.synth_outdoor_scene.argtypes = [U, D, D, D, I, I, D, D, D, D, D, D, P]
            lib.synth_outdoor_scene.restype = I
            lib.synth_trajectory.argtypes = [U, P, I, I, D, D, D, D, I, P]
            lib.synth_trajectory.restype = I
            lib.synth_cast.argtypes = [P, I, P, P]
            lib.synth_cast.restype = D
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def prim(kind: int, *params: float) -> np.ndarray:
    row = np.zeros(NPAR, np.float64)
    row[0] = kind
    row[1:1 + len(params)] = params
    return row


def scene(*rows: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.stack(rows).astype(np.float64))


def room_scene(seed: int, size=(10.0, 10.0, 3.0), n_boxes=40, n_spheres=20,
               edge=(0.2, 1.5), radius=(0.1, 0.5)) -> np.ndarray:
    out = np.zeros((1 + n_boxes + n_spheres, NPAR), np.float64)
    n = _load().synth_room_scene(seed, *size, n_boxes, n_spheres, *edge, *radius, _ptr(out))
    return out[:n]


def outdoor_scene(seed: int, size=(40.0, 40.0, 5.0), n_boxes=200, n_cyl=50,
                  edge=(0.2, 1.5), radius=(0.1, 0.5), height=(1.0, 5.0)) -> np.ndarray:
    out = np.zeros((1 + n_boxes + n_cyl, NPAR), np.float64)
    n = _load().synth_outdoor_scene(seed, *size, n_boxes, n_cyl, *edge, *radius, *height, _ptr(out))
    return out[:n]


def trajectory(seed: int, prims: np.ndarray, n_samples: int, n_way=8, xy=(1.5, 8.5),
               z=1.5, clear=0.3) -> np.ndarray:
    """(n_samples, 4, 4) camera-to-world poses on a seeded Catmull-Rom path."""
    prims = np.ascontiguousarray(prims, np.float64)
    out = np.zeros((n_samples, 4, 4), np.float64)
    rc = _load().synth_trajectory(seed, _ptr(prims), len(prims), n_way, xy[0], xy[1], z, clear,
                                  n_samples, _ptr(out))
    if rc < 0:
        raise RuntimeError(f"synth_trajectory failed ({rc})")
    return out


def render_pinhole(prims: np.ndarray, T: np.ndarray, fu, fv, cu, cv, W, H, sigma_z2=0.0,
                   invalid_frac=0.0, max_depth=math.inf, seed=0, frame=0) -> np.ndarray:
    prims = np.ascontiguousarray(prims, np.float64)
    T = np.ascontiguousarray(T, np.float64).reshape(16)
    out = np.zeros((H, W), np.float32)
    _load().synth_render_pinhole(_ptr(prims), len(prims), _ptr(T), fu, fv, cu, cv, W, H, sigma_z2,
                                 invalid_frac, max_depth, seed, frame, _ptr(out))
    return out


def render_lidar(prims: np.ndarray, T: np.ndarray, n_az, n_el, theta_start, phi_start, el_fov,
                 min_range, max_range, sigma=0.0, seed=0, frame=0) -> np.ndarray:
    prims = np.ascontiguousarray(prims, np.float64)
    T = np.ascontiguousarray(T, np.float64).reshape(16)
    out = np.zeros((n_el, n_az), np.float32)
    _load().synth_render_lidar(_ptr(prims), len(prims), _ptr(T), n_az, n_el, theta_start,
                               phi_start, el_fov, min_range, max_range, sigma, seed, frame,
                               _ptr(out))
    return out


def cast(prims: np.ndarray, o, d) -> float:
    prims = np.ascontiguousarray(prims, np.float64)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    return _load().synth_cast(_ptr(prims), len(prims), _ptr(o), _ptr(d))


from .configs import *  # noqa: E402,F401,F403
