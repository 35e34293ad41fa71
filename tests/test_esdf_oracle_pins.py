"""Pins of the ESDF oracle (Sec. IV-C) against brute force and closed forms.

The TSDF inputs are written directly from signed distance functions of
planes and spheres (no integration involved), so the site set is known; the
exact Euclidean distance transform over the observed voxels is computed by
brute force (every voxel against every site) and is the reference.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import ESDF_INSIDE, ESDF_OBS, ESDF_PAR, ESDF_SITE, esdf_offsets
from tests.esdf_inputs import V, brute_edt2, occupancy_region, tsdf_region

pytestmark = pytest.mark.filterwarnings("ignore")


def run(keys, D, W, eps, max_dist, changed=None, e=None):
    e = e or oracle.EsdfOracle(float(V), eps, 1e-4, max_dist)
    it = e.update(keys, D, W, changed)
    k, st = e.export()
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    np.testing.assert_array_equal(k, keys[order])
    return e, st, order, it


def check_parents_are_sites(st, g_sorted, site_set):
    par = (st & ESDF_PAR) != 0
    pg = g_sorted + esdf_offsets(st)
    for p in pg[par].reshape(-1, 3)[:: max(1, par.sum() // 20000)]:
        assert tuple(p) in site_set


def test_plane_equals_brute_force():
    """Plane z = 0.43 m: every observed voxel's distance is its exact
    distance (in voxels) to the nearest site, across block borders; the
    side (inside = D < 0) follows the TSDF sign."""
    eps = float(V)
    keys, D, W, g = tsdf_region((0, 0, 0), (3, 3, 4), lambda c: c[..., 2] - 0.43)
    e, st, order, it = run(keys, D, W, eps, 40)
    site = np.abs(D) <= np.float32(eps)
    exact = brute_edt2(g, site, W > 0)
    d2 = (esdf_offsets(st) ** 2).sum(-1)
    assert np.all((st & ESDF_PAR) != 0)
    np.testing.assert_array_equal(d2, exact[order])
    np.testing.assert_array_equal((st & ESDF_SITE) != 0, site[order])
    np.testing.assert_array_equal((st & ESDF_INSIDE) != 0, (D < 0)[order])
    assert d2.max() >= 20 ** 2 and it >= 3  # distances cross several blocks


def test_sphere_close_to_brute_force():
    """Sphere r = 0.52 m: parent propagation reaches every voxel, each parent
    is a site and no distance is below the exact one.  Propagation keeps,
    per voxel, one of the sites handed on by its six neighbours, so near a
    curved surface it can miss the nearest site: a site one diagonal step
    away (sqrt 2) that no axis neighbour carries is replaced by one two axis
    steps away, an excess of 2 - sqrt 2.  The excess stays within that and
    at least 93 % of the voxels are exact."""
    eps = float(V)
    ctr = np.array([0.83, 0.77, 0.91])
    keys, D, W, g = tsdf_region((0, 0, 0), (4, 4, 4),
                                lambda c: np.linalg.norm(c - ctr, axis=-1) - 0.52)
    e, st, order, _ = run(keys, D, W, eps, 60)
    site = np.abs(D) <= np.float32(eps)
    exact = brute_edt2(g, site, W > 0)[order]
    d2 = (esdf_offsets(st) ** 2).sum(-1)
    assert np.all((st & ESDF_PAR) != 0)
    assert np.all(d2 >= exact)
    excess = np.sqrt(d2) - np.sqrt(exact)
    assert excess.max() <= 2 - np.sqrt(2) + 1e-9
    assert np.mean(d2 == exact) >= 0.93
    check_parents_are_sites(st, g[order], set(map(tuple, g[site].reshape(-1, 3))))


def test_max_distance():
    """Voxels farther than max_dist from every site keep no parent; the rest
    are exact (plane)."""
    eps = float(V)
    keys, D, W, g = tsdf_region((0, 0, 0), (2, 2, 4), lambda c: c[..., 2] - 0.43)
    _, st, order, _ = run(keys, D, W, eps, 5)
    exact = brute_edt2(g, np.abs(D) <= np.float32(eps), W > 0)[order]
    par = (st & ESDF_PAR) != 0
    np.testing.assert_array_equal(par, exact <= 25)
    np.testing.assert_array_equal((esdf_offsets(st) ** 2).sum(-1)[par], exact[par])
    assert np.all(st[~par] == ESDF_OBS) or np.all((st[~par] & ESDF_OBS) != 0)


def test_incremental_move_equals_fresh():
    """A plane at z = 0.43 m, then the part with x < 0.6 m moved to 0.97 m:
    updating with only the changed blocks clears the children of the
    vanished sites and gives the same distances and flags as computing the
    second TSDF from scratch (a voxel may keep another parent at the same
    distance: ties keep the parent found first); every parent is a current
    site and no distance is below brute force."""
    eps = float(V)
    f1 = lambda c: c[..., 2] - 0.43  # noqa: E731
    f2 = lambda c: np.where(c[..., 0] < 0.6, c[..., 2] - 0.97, c[..., 2] - 0.43)  # noqa: E731
    keys, D1, W, g = tsdf_region((0, 0, 0), (3, 2, 4), f1)
    _, D2, _, _ = tsdf_region((0, 0, 0), (3, 2, 4), f2)
    changed = np.any(D1 != D2, axis=1)
    assert 0 < changed.sum() < len(keys)
    e, _, _, _ = run(keys, D1, W, eps, 40)
    _, st_inc, order, _ = run(keys, D2, W, eps, 40, changed=changed, e=e)
    assert e.counters()["cleared"] > 0
    _, st_fresh, _, _ = run(keys, D2, W, eps, 40)
    flags = ESDF_OBS | ESDF_SITE | ESDF_PAR | ESDF_INSIDE
    np.testing.assert_array_equal(st_inc & flags, st_fresh & flags)
    np.testing.assert_array_equal((esdf_offsets(st_inc) ** 2).sum(-1),
                                  (esdf_offsets(st_fresh) ** 2).sum(-1))
    site = np.abs(D2) <= np.float32(eps)
    exact = brute_edt2(g, site, W > 0)[order]
    d2 = (esdf_offsets(st_inc) ** 2).sum(-1)
    assert np.all(d2 >= exact) and np.mean(d2 == exact) >= 0.9
    check_parents_are_sites(st_inc, g[order], set(map(tuple, g[site].reshape(-1, 3))))


def test_unknown_voxels_stay_unknown():
    """Voxels with weight 0 are unknown (state 0) and pass nothing on: a
    fully unknown slab between two observed slabs keeps the far slab's
    voxels from the near slab's sites."""
    eps = float(V)
    obs = lambda c: (c[..., 2] < 0.8) | (c[..., 2] > 1.2)  # noqa: E731
    keys, D, W, g = tsdf_region((0, 0, 0), (2, 2, 4), lambda c: c[..., 2] - 0.43, observed=obs)
    _, st, order, _ = run(keys, D, W, eps, 60)
    unknown = (W == 0)[order]
    assert unknown.any()
    assert np.all(st[unknown] == 0)
    far = (g[order][..., 2] * float(V) > 1.2)
    assert np.all((st[far] & ESDF_PAR) == 0)  # no site beyond the unknown slab


def test_bad_parameters():
    with pytest.raises(ValueError):
        oracle.EsdfOracle(float(V), float(V), 1e-4, 256)
    with pytest.raises(ValueError):
        oracle.EsdfOracle(float(V), -1.0, 1e-4, 10)


# ------------------------------------------------ occupancy layers (Sec. IV-C)
# An occupancy voxel is a site if it is occupied (log-odds > 0) and one of
# its six face neighbours is free (log-odds < 0); log-odds 0 is unknown.

def run_occ(keys, L, max_dist, changed=None, e=None):
    e = e or oracle.EsdfOracle(float(V), 0.0, 0.0, max_dist, occupancy=True)
    it = e.update(keys, L, np.zeros_like(L), changed)
    k, st = e.export()
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    np.testing.assert_array_equal(k, keys[order])
    return e, st, order, it


def test_occupancy_half_space_equals_brute_force():
    """Occupied below z = 0.4 m (voxels gz < 8, a block face), free above:
    the sites are exactly the occupied layer gz = 7 (its +z neighbour is
    free), inside = occupied, and every voxel's distance is its exact
    distance to that layer, across block borders and on both sides."""
    keys, L, g = occupancy_region((0, 0, 0), (3, 3, 4), lambda c: c[..., 2] < 0.4)
    _, st, order, it = run_occ(keys, L, 40)
    gz = g[order][..., 2]
    np.testing.assert_array_equal((st & ESDF_SITE) != 0, gz == 7)
    np.testing.assert_array_equal((st & ESDF_INSIDE) != 0, gz < 8)
    assert np.all((st & ESDF_OBS) != 0) and np.all((st & ESDF_PAR) != 0)
    exact = brute_edt2(g, g[..., 2] == 7, np.ones(L.shape, bool))[order]
    np.testing.assert_array_equal((esdf_offsets(st) ** 2).sum(-1), exact)
    assert exact.max() >= 20 ** 2 and it >= 3


def test_occupancy_box_close_to_brute_force():
    """An occupied box of voxels [10, 17]^3 in free space: the sites are the
    box's surface voxels (a coordinate at 10 or 17); no distance is below
    the exact one, the excess stays within 2 - sqrt 2 and most voxels are
    exact."""
    inbox = lambda c: np.all((c >= 10 * float(V)) & (c < 18 * float(V)), axis=-1)  # noqa: E731
    keys, L, g = occupancy_region((0, 0, 0), (4, 4, 4), inbox)
    _, st, order, _ = run_occ(keys, L, 60)
    gs = g[order]
    box = np.all((gs >= 10) & (gs <= 17), -1)
    shell = box & np.any((gs == 10) | (gs == 17), -1)
    np.testing.assert_array_equal((st & ESDF_SITE) != 0, shell)
    np.testing.assert_array_equal((st & ESDF_INSIDE) != 0, box)
    exact = brute_edt2(gs, shell, np.ones(shell.shape, bool))
    d2 = (esdf_offsets(st) ** 2).sum(-1)
    assert np.all((st & ESDF_PAR) != 0)
    assert np.all(d2 >= exact)
    assert (np.sqrt(d2) - np.sqrt(exact)).max() <= 2 - np.sqrt(2) + 1e-9
    assert np.mean(d2 == exact) >= 0.9
    check_parents_are_sites(st, gs, set(map(tuple, gs[shell].reshape(-1, 3))))


def test_occupancy_unknown_neighbours_make_no_sites():
    """Occupied below z = 0.4 m, unknown (log-odds 0) for 0.4 <= z < 0.6 m,
    free above, and no blocks beyond x = 0.8 m: no occupied voxel touches a
    free one, so there is no site and no parent; unknown voxels stay 0."""
    keys, L, g = occupancy_region((0, 0, 0), (2, 2, 4), lambda c: c[..., 2] < 0.4,
                                  known=lambda c: (c[..., 2] < 0.4) | (c[..., 2] >= 0.6))
    _, st, order, _ = run_occ(keys, L, 40)
    assert not np.any(st & ESDF_SITE) and not np.any(st & ESDF_PAR)
    np.testing.assert_array_equal(st == 0, (L == 0)[order])


def test_occupancy_incremental_across_block_face():
    """Occupied below z = 0.4 m, then below z = 0.5 m: only the blocks above
    the face z = 0.4 m change, yet the old sites (gz = 7, in the unchanged
    blocks below) stop being sites because their +z neighbours are now
    occupied.  The incremental update equals a fresh computation of the
    second layer (flags and distances) and is exact against brute force."""
    keys, L1, g = occupancy_region((0, 0, 0), (3, 2, 4), lambda c: c[..., 2] < 0.4)
    _, L2, _ = occupancy_region((0, 0, 0), (3, 2, 4), lambda c: c[..., 2] < 0.5)
    changed = np.any(L1 != L2, axis=1)
    assert np.all(keys[changed][:, 2] == 1) and not np.any(changed[keys[:, 2] == 0])
    e, _, _, _ = run_occ(keys, L1, 40)
    _, st_inc, order, _ = run_occ(keys, L2, 40, changed=changed, e=e)
    assert e.counters()["cleared"] > 0
    _, st_fresh, _, _ = run_occ(keys, L2, 40)
    flags = ESDF_OBS | ESDF_SITE | ESDF_PAR | ESDF_INSIDE
    np.testing.assert_array_equal(st_inc & flags, st_fresh & flags)
    d2 = (esdf_offsets(st_inc) ** 2).sum(-1)
    np.testing.assert_array_equal(d2, (esdf_offsets(st_fresh) ** 2).sum(-1))
    gz = g[order][..., 2]
    np.testing.assert_array_equal((st_inc & ESDF_SITE) != 0, gz == 9)
    np.testing.assert_array_equal(d2, brute_edt2(g, g[..., 2] == 9, np.ones(L2.shape, bool))[order])
