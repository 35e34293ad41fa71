"""Workload recipes (seeded, synthetic) for the TSDF integration path.

Each recipe returns plain numpy data: sensor intrinsics as dicts, camera- or
LiDAR-to-world poses as (4, 4) float64 arrays and depth / range images as
float32 arrays.  The recipes are the stand-ins for the paper's datasets
(Replica / Redwood RGB-D rooms, a 64-beam spinning LiDAR; Sec. V) and carry
the sizes of the paper's workloads at the resolutions used here.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import (BOX, PLANE, SPHERE, outdoor_scene, prim, render_lidar, render_pinhole,
               room_scene, scene, trajectory)

__all__ = ["Frame", "Workload", "pinhole", "lidar64", "config_tiny", "config_room",
           "config_rig", "config_serving_maps", "serving_arrivals", "render_frame",
           "color_image", "room_colors", "cached"]

_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".synth_cache")


def pinhole(W, H, f, cu=None, cv=None, fv=None):
    return {"kind": "pinhole", "fu": float(f), "fv": float(f if fv is None else fv),
            "cu": float((W - 1) / 2 if cu is None else cu),
            "cv": float((H - 1) / 2 if cv is None else cv), "width": int(W), "height": int(H)}


def lidar64(n_az=1024, n_el=64, fov_deg=45.0, min_range=0.5, max_range=30.0):
    """Spinning LiDAR, full azimuth circle, symmetric vertical FoV."""
    return {"kind": "lidar", "n_az": int(n_az), "n_el": int(n_el), "theta_start": -math.pi,
            "phi_start": math.radians(90.0 - fov_deg / 2), "el_fov": math.radians(fov_deg),
            "min_range": float(min_range), "max_range": float(max_range)}


@dataclass
class Frame:
    sensor: dict
    T: np.ndarray          # (4,4) float64 sensor-to-world
    depth: np.ndarray      # float32 (H, W) z-depth or (n_el, n_az) range
    map_id: int = 0


@dataclass
class Workload:
    name: str
    voxel_size: float
    truncation_voxels: int
    max_weight: float
    frames: list = field(default_factory=list)


def render_frame(prims, sensor, T, noise: dict, seed: int, frame: int) -> np.ndarray:
    if sensor["kind"] == "pinhole":
        return render_pinhole(prims, T, sensor["fu"], sensor["fv"], sensor["cu"], sensor["cv"],
                              sensor["width"], sensor["height"], noise.get("sigma_z2", 0.0),
                              noise.get("invalid_frac", 0.0), noise.get("max_depth", math.inf),
                              seed, frame)
    return render_lidar(prims, T, sensor["n_az"], sensor["n_el"], sensor["theta_start"],
                        sensor["phi_start"], sensor["el_fov"], sensor["min_range"],
                        sensor["max_range"], noise.get("sigma", 0.0), seed, frame)


def color_image(sensor, T, depth, seed: int, frame: int) -> np.ndarray:
    """Colour image registered to a pinhole depth image: uint32 [H, W], r in
    the low byte, then g, b (top byte 0).  The colour is a smooth procedural
    texture of the world point the pixel sees (back-projected from its
    depth), so views of one surface agree, plus a seeded per-pixel jitter of
    up to +-3 levels per channel (sensor noise); pixels without a valid
    depth get a random colour."""
    H, W = sensor["height"], sensor["width"]
    jj, ii = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    d = depth.astype(np.float64)
    ok = np.isfinite(d) & (d > 0)
    d = np.where(ok, d, 1.0)
    pc = np.stack([(ii - sensor["cu"]) / sensor["fu"] * d, (jj - sensor["cv"]) / sensor["fv"] * d, d])
    pw = np.einsum("ij,jhw->ihw", T[:3, :3], pc) + T[:3, 3, None, None]
    x, y, z = pw
    tex = np.stack([128 + 100 * np.sin(3.1 * x + 1.3 * z), 128 + 100 * np.sin(2.3 * y - 0.7 * x),
                    128 + 100 * np.cos(1.7 * z + 2.9 * y)])
    rng = np.random.default_rng([seed, frame, 7])
    tex = np.rint(tex) + rng.integers(-3, 4, size=tex.shape)
    tex = np.where(ok[None], tex, rng.integers(0, 256, size=tex.shape))
    c = np.clip(tex, 0, 255).astype(np.uint32)
    return (c[0] | (c[1] << 8) | (c[2] << 16)).astype(np.uint32)


def room_colors(w: Workload, seed: int = 3, use_cache: bool = True) -> np.ndarray:
    """Colour images (uint32 [n, H, W]) registered to every frame of a
    pinhole workload, by color_image."""
    def make():
        return np.stack([color_image(f.sensor, f.T, f.depth, seed, i)
                         for i, f in enumerate(w.frames)])
    key = f"colors:{w.name}:{seed}:{hashlib.sha1(w.frames[0].depth.tobytes()).hexdigest()[:12]}"
    return cached(key, make) if use_cache else make()


def cached(key: str, fn):
    """Memoise an array-returning recipe step on disk (inputs only)."""
    os.makedirs(_CACHE, exist_ok=True)
    path = os.path.join(_CACHE, hashlib.sha1(key.encode()).hexdigest()[:20] + ".npy")
    if os.path.exists(path):
        return np.load(path)
    arr = fn()
    np.save(path + ".tmp.npy", arr)
    os.replace(path + ".tmp.npy", path)
    return arr


def config_tiny() -> Workload:
    """64x48 pinhole (f=50, c=(32,24)), identity pose; plane z=2 m plus a
    sphere r=0.3 m at (0.2, 0.1, 1.5) m; exact ray casting, no noise;
    voxel 0.05 m, truncation 4 voxels, max weight 100."""
    prims = tiny_scene()
    cam = pinhole(64, 48, 50.0, 32.0, 24.0)
    T = np.eye(4)
    d = render_frame(prims, cam, T, {}, 0, 0)
    return Workload("tiny 64x48 plane+sphere", 0.05, 4, 100.0, [Frame(cam, T, d)])


def tiny_scene() -> np.ndarray:
    return scene(prim(PLANE, 0.0, 0.0, 1.0, 2.0), prim(SPHERE, 0.2, 0.1, 1.5, 0.3))


ROOM_NOISE = {"sigma_z2": 0.0012, "invalid_frac": 0.05, "max_depth": 5.0}


def config_room(n_frames: int = 300, seed: int = 2, W=640, H=480, f=525.0,
                noise: dict | None = None, use_cache: bool = True) -> Workload:
    """Seeded 10x10x3 m room: 40 boxes (edges 0.2-1.5 m), 20 spheres
    (r 0.1-0.5 m); camera on a Catmull-Rom path through 8 waypoints at 1.5 m
    height; 640x480 pinhole, f=525, c=(319.5, 239.5); noise N(0,(0.0012 z^2)^2),
    5 % invalid pixels, depth > 5 m invalid; voxel 0.02 m, truncation 4 voxels,
    max weight 100."""
    noise = ROOM_NOISE if noise is None else noise
    prims = room_scene(seed)
    Ts = trajectory(seed, prims, n_frames)
    cam = pinhole(W, H, f, (W - 1) / 2, (H - 1) / 2)
    key = f"room:{seed}:{n_frames}:{W}x{H}:{f}:{sorted(noise.items())}"

    def make():
        return np.stack([render_frame(prims, cam, Ts[i], noise, seed, i) for i in range(n_frames)])

    depths = cached(key, make) if use_cache else make()
    frames = [Frame(cam, Ts[i], depths[i]) for i in range(n_frames)]
    return Workload(f"room 10x10x3 m, {n_frames} frames {W}x{H}", 0.02, 4, 100.0, frames)


RIG_CAMS = [pinhole(640, 480, 525.0), pinhole(640, 480, 525.0),
            pinhole(848, 480, 525.0 * 848 / 640), pinhole(1280, 720, 1050.0)]
RIG_LIDAR_NOISE = {"sigma": 0.02}


def rig_poses(T_rig: np.ndarray):
    """Four cameras at 0/90/180/270 deg yaw about the rig's vertical axis,
    10 cm from the rig origin, and a LiDAR at the origin (z up)."""
    out = []
    fwd = T_rig[:3, 2]
    for k in range(4):
        a = k * math.pi / 2
        c, s = math.cos(a), math.sin(a)
        Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        T = np.eye(4)
        T[:3, :3] = Rz @ T_rig[:3, :3]
        T[:3, 3] = T_rig[:3, 3] + 0.1 * (Rz @ fwd)
        out.append(T)
    # LiDAR: z up, x along the rig heading
    TL = np.eye(4)
    TL[:3, 0] = fwd
    TL[:3, 2] = [0.0, 0.0, 1.0]
    TL[:3, 1] = np.cross(TL[:3, 2], TL[:3, 0])
    TL[:3, 3] = T_rig[:3, 3]
    out.append(TL)
    return out


def config_rig(n_steps: int = 200, seed: int = 4, use_cache: bool = True) -> Workload:
    """Outdoor 40x40x5 m scene (200 boxes, 50 vertical cylinders, ground
    plane); rig of 4 pinhole cameras (640x480, 640x480, 848x480, 1280x720) at
    90 deg yaw offsets and a 1024x64 LiDAR (-22.5..22.5 deg, 0.5-30 m,
    N(0, 0.02^2)); rig on a seeded path at 1.5 m; voxel 0.05 m, truncation 4
    voxels.  Frames are ordered cam0..cam3, lidar within each step."""
    prims = outdoor_scene(seed)
    Ts = trajectory(seed, prims, n_steps, n_way=8, xy=(4.0, 36.0), z=1.5, clear=0.3)
    lid = lidar64()
    frames = []
    for s in range(n_steps):
        poses = rig_poses(Ts[s])
        for k, cam in enumerate(RIG_CAMS):
            key = f"rig:{seed}:{n_steps}:{s}:{k}"
            d = cached(key, lambda: render_frame(prims, cam, poses[k], ROOM_NOISE, seed,
                                                 s * 8 + k)) if use_cache else \
                render_frame(prims, cam, poses[k], ROOM_NOISE, seed, s * 8 + k)
            frames.append(Frame(cam, poses[k], d))
        key = f"rig:{seed}:{n_steps}:{s}:lidar"
        d = cached(key, lambda: render_frame(prims, lid, poses[4], RIG_LIDAR_NOISE, seed,
                                             s * 8 + 4)) if use_cache else \
            render_frame(prims, lid, poses[4], RIG_LIDAR_NOISE, seed, s * 8 + 4)
        frames.append(Frame(lid, poses[4], d))
    return Workload(f"rig outdoor 40x40x5 m, {n_steps} steps x 5 frames", 0.05, 4, 100.0, frames)


SERVING_SENSORS = [pinhole(320, 240, 262.5), pinhole(640, 480, 525.0),
                   pinhole(1280, 720, 1050.0), lidar64()]


def config_serving_maps(n_maps: int = 16, seed: int = 5):
    """Per-map voxel size drawn from {0.02, 0.05, 0.1} m and a per-map seeded
    room scene as in the room recipe."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([0.02, 0.05, 0.1], size=n_maps)
    maps = []
    for m in range(n_maps):
        prims = room_scene(seed * 1000 + m)
        maps.append({"voxel_size": float(sizes[m]), "truncation_voxels": 4,
                     "max_weight": 100.0, "prims": prims, "seed": seed * 1000 + m})
    return maps


def serving_arrivals(n_maps: int = 16, rate_hz: float = 30.0, duration_s: float = 60.0,
                     seed: int = 5):
    """Per-map Poisson arrival times and sensor choices: list of
    (t, map_id, sensor_index) sorted by time."""
    rng = np.random.default_rng(seed + 1)
    out = []
    for m in range(n_maps):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rate_hz)
            if t >= duration_s:
                break
            out.append((t, m, int(rng.integers(0, len(SERVING_SENSORS)))))
    out.sort()
    return out
