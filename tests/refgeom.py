"""Independent FP64 geometry used by the oracle pins (test-only helpers).

Nothing here is copied from the oracle or the CUDA path: it is a direct,
vectorised restatement of the geometry (pinhole / spherical projection, a
slab test for ray-segment / block intersection, bilinear sampling) used to
derive expected values for closed-form scenes and brute-force checks.
Decisions that land within a small margin of a boundary are reported as
ambiguous so that tests can leave them out.
"""
from __future__ import annotations

import math

import numpy as np


def voxel_centres(keys: np.ndarray, v: float) -> np.ndarray:
    """(n, 512, 3) FP64 voxel centres of blocks `keys` (voxel x fastest)."""
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    g = keys[:, None, :].astype(np.int64) * 8 + loc[None]
    return (g + 0.5) * float(v)


def to_sensor(T: np.ndarray, pL: np.ndarray) -> np.ndarray:
    R, t = T[:3, :3], T[:3, 3]
    return (pL - t) @ R


def pinhole_pixel(cam: dict, pC: np.ndarray, margin: float = 1e-5):
    """Nearest pixel of each point and an `ok` mask of unambiguous decisions.

    Returns (i, j, inside, ok): inside = z > 0 and pixel in image; ok = all
    rounding and border decisions are at least `margin` px from a tie."""
    z = pC[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = cam["fu"] * pC[..., 0] / z + cam["cu"] + 0.5
        v = cam["fv"] * pC[..., 1] / z + cam["cv"] + 0.5
    W, H = cam["width"], cam["height"]
    pos = z > 0
    i = np.floor(np.where(pos, u, -1)).astype(np.int64)
    j = np.floor(np.where(pos, v, -1)).astype(np.int64)
    inside = pos & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    fu, fv = u - np.floor(u), v - np.floor(v)
    ok = (~pos) | ((np.minimum(fu, 1 - fu) > margin) & (np.minimum(fv, 1 - fv) > margin)
                   & (np.abs(u) > margin) & (np.abs(u - W) > margin)
                   & (np.abs(v) > margin) & (np.abs(v - H) > margin))
    ok &= np.abs(z) > 1e-6
    return i, j, inside, ok


def segment_cells(o: np.ndarray, d: np.ndarray, s0: float, s1: float, B: float,
                  eps_cell: float = 1e-4, eps_s: float = 1e-5):
    """Blocks (global integer coords) met by the segment o + s d, s in
    [s0, s1], by a slab test over the candidate blocks around the segment.

    Returns (definite, possible) as sets of tuples: `definite` holds the blocks
    met even when every block is shrunk by eps_cell (block units) and the
    segment by eps_s; `possible` holds those met when both are grown."""
    out = []
    for grow in (-1.0, 1.0):
        a, b = s0 - grow * eps_s, s1 + grow * eps_s
        p0, p1 = (o + a * d) / B, (o + b * d) / B
        lo = np.floor(np.minimum(p0, p1)).astype(np.int64) - 1
        hi = np.floor(np.maximum(p0, p1)).astype(np.int64) + 1
        gx, gy, gz = np.meshgrid(*[np.arange(lo[k], hi[k] + 1) for k in range(3)], indexing="ij")
        cells = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)
        cmin = cells - grow * eps_cell
        cmax = cells + 1 + grow * eps_cell
        D = p1 - p0
        tlo = np.zeros(len(cells))
        thi = np.ones(len(cells))
        for k in range(3):
            if abs(D[k]) < 1e-300:
                inside = (p0[k] >= cmin[:, k]) & (p0[k] <= cmax[:, k])
                thi = np.where(inside, thi, -1.0)
                continue
            t1 = (cmin[:, k] - p0[k]) / D[k]
            t2 = (cmax[:, k] - p0[k]) / D[k]
            tlo = np.maximum(tlo, np.minimum(t1, t2))
            thi = np.minimum(thi, np.maximum(t1, t2))
        hit = tlo <= thi
        out.append({tuple(c) for c in cells[hit]})
    return out[0], out[1]


def pinhole_band_blocks(cam: dict, T: np.ndarray, depth: np.ndarray, tau: float, B: float):
    R, t = T[:3, :3], T[:3, 3]
    definite, possible = set(), set()
    for j in range(cam["height"]):
        for i in range(cam["width"]):
            d = float(depth[j, i])
            if not (d > 0 and math.isfinite(d)):
                continue
            r = np.array([(i - cam["cu"]) / cam["fu"], (j - cam["cv"]) / cam["fv"], 1.0])
            a, b = segment_cells(t, R @ r, max(d - tau, 0.0), d + tau, B)
            definite |= a
            possible |= b
    return definite, possible


def lidar_beam(lid: dict, k: int, j: int) -> np.ndarray:
    th = lid["theta_start"] + (k + 0.5) * 2 * math.pi / lid["n_az"]
    ph = lid["phi_start"] + (j + 0.5) * lid["el_fov"] / lid["n_el"]
    return np.array([math.sin(ph) * math.cos(th), math.sin(ph) * math.sin(th), math.cos(ph)])


def lidar_band_blocks(lid: dict, T: np.ndarray, rng: np.ndarray, tau: float, B: float):
    R, t = T[:3, :3], T[:3, 3]
    definite, possible = set(), set()
    for j in range(lid["n_el"]):
        for k in range(lid["n_az"]):
            d = float(rng[j, k])
            if not (lid["min_range"] <= d <= lid["max_range"]):
                continue
            a, b = segment_cells(t, R @ lidar_beam(lid, k, j), max(d - tau, 0.0), d + tau, B)
            definite |= a
            possible |= b
    return definite, possible


def lidar_coords(lid: dict, pC: np.ndarray):
    """Continuous image coordinates (u, v) of Eq. 3 with theta = atan2(y, x)
    and phi = acos(z / r); u in [0, n_az) wraps with the azimuth."""
    x, y, z = pC[..., 0], pC[..., 1], pC[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    th = np.arctan2(y, x)
    ph = np.arccos(np.clip(z / r, -1, 1))
    alpha = lid["n_az"] / (2 * math.pi)
    beta = lid["n_el"] / lid["el_fov"]
    u = (th - lid["theta_start"]) * alpha
    v = (ph - lid["phi_start"]) * beta
    return u, v, r


def lidar_bilinear(lid: dict, rng: np.ndarray, u: np.ndarray, v: np.ndarray, guard: float,
                   margin: float = 1e-3):
    """Guarded bilinear sample at (u, v): returns (d, valid, ok) where valid =
    four valid neighbours within `guard` of each other, ok = no decision
    within `margin` of a tie."""
    n_az, n_el = lid["n_az"], lid["n_el"]
    uu, vv = u - 0.5, v - 0.5
    k0 = np.floor(uu).astype(np.int64)
    j0 = np.floor(vv).astype(np.int64)
    fx, fy = uu - k0, vv - j0
    inrow = (j0 >= 0) & (j0 <= n_el - 2)
    jc = np.clip(j0, 0, n_el - 2)
    ka = np.mod(k0, n_az)
    kb = np.mod(k0 + 1, n_az)
    d00, d10 = rng[jc, ka], rng[jc, kb]
    d01, d11 = rng[jc + 1, ka], rng[jc + 1, kb]
    quad = np.stack([d00, d10, d01, d11], -1).astype(np.float64)
    allvalid = np.all((quad >= lid["min_range"]) & (quad <= lid["max_range"]), -1)
    spread = quad.max(-1) - quad.min(-1)
    valid = inrow & allvalid & (spread <= guard)
    d = (1 - fy) * ((1 - fx) * d00 + fx * d10) + fy * ((1 - fx) * d01 + fx * d11)
    ok = (np.minimum(fx, 1 - fx) > margin) & (np.minimum(fy, 1 - fy) > margin)
    ok &= np.abs(spread - guard) > 1e-6
    return d, valid, ok
