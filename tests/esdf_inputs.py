"""TSDF layers written directly from signed distance functions, and the
brute-force Euclidean distance transform: inputs and references for the
ESDF tests (no method arithmetic)."""
from __future__ import annotations

import numpy as np

V = np.float32(0.05)


def tsdf_region(lo, hi, sdf, tau=4 * 0.05, observed=None):
    """TSDF blocks lo <= key < hi (block coords) with D = clip(sdf(centre),
    -tau, tau) and W = 1 (0 where observed(centre) is False)."""
    keys = np.array([(x, y, z) for x in range(lo[0], hi[0]) for y in range(lo[1], hi[1])
                     for z in range(lo[2], hi[2])], np.int32)
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    g = keys[:, None, :] * 8 + loc[None]
    c = (g + 0.5) * float(V)
    D = np.clip(sdf(c), -tau, tau).astype(np.float32)
    W = np.ones_like(D)
    if observed is not None:
        W[~observed(c)] = 0.0
    return keys, D, W, g


def brute_edt2(g, site_mask, obs_mask, chunk=512):
    """Exact squared distance (voxels) from every voxel to the nearest site."""
    sites = g[site_mask].astype(np.int64)
    pts = g.reshape(-1, 3).astype(np.int64)
    out = np.full(len(pts), np.iinfo(np.int64).max, np.int64)
    for s in range(0, len(pts), chunk):
        d = ((pts[s:s + chunk, None, :] - sites[None]) ** 2).sum(-1)
        out[s:s + chunk] = d.min(1)
    return out.reshape(g.shape[:-1])


def occupancy_region(lo, hi, occupied, known=None, l_occ=0.85, l_free=-0.4):
    """Occupancy blocks lo <= key < hi (block coords): log-odds l_occ where
    occupied(centre), l_free elsewhere, 0 (unknown) where known(centre) is
    False."""
    keys = np.array([(x, y, z) for x in range(lo[0], hi[0]) for y in range(lo[1], hi[1])
                     for z in range(lo[2], hi[2])], np.int32)
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    g = keys[:, None, :] * 8 + loc[None]
    c = (g + 0.5) * float(V)
    L = np.where(occupied(c), np.float32(l_occ), np.float32(l_free)).astype(np.float32)
    if known is not None:
        L[~known(c)] = 0.0
    return keys, L, g

