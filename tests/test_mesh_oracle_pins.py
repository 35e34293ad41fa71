"""Pins of the marching-cubes oracle against closed forms and topology.

TSDF inputs come from signed distance functions (tests/esdf_inputs.py).  A
plane gives vertices exactly on it and a known area; a sphere inside the
region gives a closed, outward-facing surface of genus 0; random fields
exercise every face ambiguity, where neighbouring cubes must still join
their polygon loops without gaps.
"""
from __future__ import annotations

from collections import Counter

import numpy as np
import pytest

import oracle
from tests.esdf_inputs import V, tsdf_region


def _edges(keys):
    """Directed triangle edges as hashable vertex-key pairs."""
    k = [tuple(map(tuple, t)) for t in keys]
    return [(t[i], t[(i + 1) % 3]) for t in k for i in range(3)]


def _area(pos):
    a = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    return 0.5 * np.linalg.norm(a, axis=1)


def test_every_case_closes():
    """Each of the 254 non-trivial cube cases yields loops over exactly the
    edges whose ends differ, every loop segment lies on one cube face, and
    each used edge is entered and left once."""
    corner = [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]
    edges = []
    for e in range(12):
        axis, u, w = e // 4, e & 1, (e >> 1) & 1
        o1, o2 = (1, 2) if axis == 0 else ((0, 2) if axis == 1 else (0, 1))
        lo = [0, 0, 0]
        lo[o1], lo[o2] = u, w
        hi = list(lo)
        hi[axis] = 1
        edges.append((corner.index(tuple(lo)), corner.index(tuple(hi)), axis, lo))
    for case in range(1, 255):
        tris = oracle.mesh_case(case)
        cut = {e for e, (a, b, _, _) in enumerate(edges) if ((case >> a) & 1) != ((case >> b) & 1)}
        used = set(tris.reshape(-1).tolist())
        assert used == cut, case
        # the polygon boundaries: directed edges not cancelled inside a fan
        cnt = Counter()
        for t in tris:
            for i in range(3):
                cnt[(t[i], t[(i + 1) % 3])] += 1
        bnd = [d for d in cnt if (d[1], d[0]) not in cnt]
        outs = Counter(a for a, _ in bnd)
        assert all(outs[e] == 1 for e in cut), case
        for a, b in bnd:  # both ends on a common cube face
            la, lb = edges[a][3], edges[b][3]
            fa = {(ax, la[ax]) for ax in range(3) if ax != edges[a][2]}
            fb = {(ax, lb[ax]) for ax in range(3) if ax != edges[b][2]}
            assert fa & fb, (case, a, b)


def test_plane_exact():
    """Plane z = 0.43 m: every vertex lies on it (linear interpolation of a
    linear field is exact) and the area is that of the plane over the meshed
    cubes, (8 n - 1)^2 voxel faces for n x n blocks."""
    keys, D, W, _ = tsdf_region((0, 0, 0), (3, 3, 2), lambda c: c[..., 2] - 0.43)
    _, k, pos = oracle.mesh_extract(keys, D, W, float(V))
    v = float(V)
    assert np.abs(pos[..., 2] - 0.43).max() < 1e-6  # FP32 TSDF values
    np.testing.assert_allclose(_area(pos).sum(), (23 * v) ** 2, rtol=1e-5)
    normals = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    assert np.all(normals[:, 2] > 0)  # facing +z, where D grows


@pytest.mark.parametrize("r", [0.31, 0.52])
def test_sphere_closed_outward(r):
    """A sphere inside the region: every directed edge has its reverse
    exactly once (closed 2-manifold), V - E + F = 2, triangles face away
    from the centre, the area is within 3 % of 4 pi r^2."""
    ctr = np.array([0.83, 0.77, 0.91])
    keys, D, W, _ = tsdf_region((0, 0, 0), (4, 4, 4), lambda c: np.linalg.norm(c - ctr, axis=-1) - r)
    _, k, pos = oracle.mesh_extract(keys, D, W, float(V))
    de = Counter(_edges(k))
    assert all(n == 1 for n in de.values())
    assert all(de[(b, a)] == 1 for a, b in de)
    nv = len({tuple(x) for x in k.reshape(-1, 4).tolist()})
    assert nv - len(de) // 2 + len(k) == 2
    normals = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    assert np.all((normals * (pos.mean(1) - ctr)).sum(1) > 0)
    np.testing.assert_allclose(_area(pos).sum(), 4 * np.pi * r * r, rtol=0.03)
    assert np.abs(np.linalg.norm(pos - ctr, axis=-1) - r).max() < 0.5 * float(V)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_field_crack_free(seed):
    """Random values (many ambiguous faces): each cube's loop boundary (its
    directed edges not cancelled inside the cube) is, segment by segment,
    the reverse of a neighbouring cube's boundary, except on the outer faces
    of the region: shared faces are resolved the same way on both sides,
    so the loops leave no gaps."""
    rng = np.random.default_rng(seed)
    field = rng.normal(size=(16, 16, 16)).astype(np.float32)
    keys, D, W, g = tsdf_region((0, 0, 0), (2, 2, 2), lambda c: np.zeros(c.shape[:-1]))
    D = field[g[..., 0], g[..., 1], g[..., 2]]
    cube, k, _ = oracle.mesh_extract(keys, D, W, float(V))
    per_cube = {}
    for c, t in zip(map(tuple, cube.tolist()), k):
        tt = [tuple(x) for x in t.tolist()]
        per_cube.setdefault(c, Counter()).update((tt[i], tt[(i + 1) % 3]) for i in range(3))
    seg = Counter()
    for cnt in per_cube.values():
        seg.update(d for d in cnt if (d[1], d[0]) not in cnt)
    assert all(n == 1 for n in seg.values())
    def on_outer_face(a, b):  # both vertex edges lie on one outer face of the region
        for ax in range(3):
            for val in (0, 15):
                if all(v[ax] == val and v[3] != ax for v in (a, b)):
                    return True
        return False
    open_segs = [d for d in seg if seg[(d[1], d[0])] != 1]
    assert all(on_outer_face(*d) for d in open_segs)
    assert len(seg) > 1000


def test_blocks_partition_and_unobserved():
    """Meshing blocks one at a time gives the same triangles as all at
    once; cubes with an unobserved corner give none."""
    ctr = np.array([0.5, 0.5, 0.5])
    obs = lambda c: c[..., 0] < 0.6  # noqa: E731
    keys, D, W, _ = tsdf_region((0, 0, 0), (2, 2, 2), lambda c: np.linalg.norm(c - ctr, axis=-1) - 0.3,
                                observed=obs)
    _, k_all, _ = oracle.mesh_extract(keys, D, W, float(V))
    parts = [oracle.mesh_extract(keys, D, W, float(V), blocks=np.arange(len(keys)) == i)[1]
             for i in range(len(keys))]
    merged = np.concatenate(parts)
    assert sorted(map(lambda t: t.tobytes(), merged)) == sorted(map(lambda t: t.tobytes(), k_all))
    # no vertex on an edge touching an unobserved voxel (centre x >= 0.6 m)
    top = k_all[..., 0] + (k_all[..., 3] == 0)  # x index of the edge's upper corner
    assert len(k_all) > 0 and np.all((top + 0.5) * float(V) < 0.6)


def test_ambiguous_face_separates_inside_corners():
    """Corners 0 and 3 (diagonal on the face z = 0) inside, the rest
    outside: the face rule keeps them apart, giving two corner triangles
    (edges 0, 4, 8 around corner 0 and 1, 5, 11 around corner 3), not
    one tube joining them."""
    tris = oracle.mesh_case(0b00001001)
    assert len(tris) == 2
    assert sorted(map(sorted, tris.tolist())) == [[0, 4, 8], [1, 5, 11]]


def test_zero_is_outside():
    """D = 0 counts as outside (inside is D < 0): for D = (z index - 8)
    voxels the vertices sit on the edges from z index 7 to 8, at t = 1."""
    keys, D, W, g = tsdf_region((0, 0, 0), (2, 2, 2), lambda c: np.zeros(c.shape[:-1]))
    D = (g[..., 2] - 8).astype(np.float32) * np.float32(V)
    _, k, pos = oracle.mesh_extract(keys, D, W, float(V))
    assert len(k) > 0
    assert np.all(k[..., 3] == 2) and np.all(k[..., 2] == 7)
    np.testing.assert_allclose(pos[..., 2], (8 + 0.5) * float(V), rtol=0, atol=1e-12)
