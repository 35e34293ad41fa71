"""GPU parity of the ESDF layer (Sec. IV-C) against the oracle, through the C
ABI.

Both sides start from the same FP32 TSDF: blocks written from signed
distance functions, or integrated by the FP64 oracle and rounded to FP32,
and imported into the GPU map with map_import.  The ESDF arithmetic is
integer, so the voxel states (flags and parent offsets) must match bit for
bit, and so must the iteration, sweep, exchange and clearing counts.  A
GPU-integrated room is checked by properties: every parent is a site of the
GPU's own layer and no distance is below the brute-force one.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from tests.esdf_inputs import V, tsdf_region

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2311_00626_gb300 as gt  # noqa: E402
from oracle import ESDF_INSIDE, ESDF_OBS, ESDF_PAR, ESDF_SITE, esdf_offsets  # noqa: E402


def _pair(v, eps, max_dist, max_blocks=1 << 14):
    g = gt.TsdfMap(float(v), max_blocks=max_blocks)
    o = oracle.EsdfOracle(float(v), eps, 1e-4, max_dist)
    return g, o


def _step(g, o, keys, D, W, changed, eps, max_dist):
    """Import the changed blocks into the GPU map, update both layers,
    compare states and counters."""
    ch = np.ones(len(keys), bool) if changed is None else changed
    g.import_blocks(keys[ch], D[ch], W[ch])
    g.esdf_update(eps, 1e-4, max_dist)
    o.update(keys, D, W, ch)
    gk, gs = g.esdf_export()
    ok, os_ = o.export()
    np.testing.assert_array_equal(gk, ok)
    bad = np.count_nonzero(gs != os_)
    assert bad == 0, f"{bad} ESDF voxel states differ"
    gc, oc = g.esdf_stats(), o.counters()
    assert gc == oc, (gc, oc)
    return gk, gs


def test_plane_and_sphere_bit_exact():
    eps = float(V)
    for sdf, lo, hi in ((lambda c: c[..., 2] - 0.43, (0, 0, 0), (3, 3, 4)),
                        (lambda c: np.linalg.norm(c - np.array([0.83, 0.77, 0.91]), axis=-1) - 0.52,
                         (0, 0, 0), (4, 4, 4)),
                        (lambda c: np.linalg.norm(c - np.array([-0.31, 0.2, -0.6]), axis=-1) - 0.4,
                         (-3, -2, -4), (1, 2, 0))):
        keys, D, W, _ = tsdf_region(lo, hi, sdf)
        g, o = _pair(V, eps, 60)
        _, st = _step(g, o, keys, D, W, None, eps, 60)
        assert np.all((st & ESDF_PAR) != 0)
        g.close()
        o.close()


def test_incremental_clear_bit_exact():
    """Moved surface: only the changed blocks are imported; the clearing of
    the vanished sites' children and the relowering match the oracle."""
    eps = float(V)
    f1 = lambda c: c[..., 2] - 0.43  # noqa: E731
    f2 = lambda c: np.where(c[..., 0] < 0.6, c[..., 2] - 0.97, c[..., 2] - 0.43)  # noqa: E731
    keys, D1, W, _ = tsdf_region((0, 0, 0), (3, 2, 4), f1)
    _, D2, _, _ = tsdf_region((0, 0, 0), (3, 2, 4), f2)
    g, o = _pair(V, eps, 40)
    _step(g, o, keys, D1, W, None, eps, 40)
    _step(g, o, keys, D2, W, np.any(D1 != D2, axis=1), eps, 40)
    assert g.esdf_stats()["cleared"] > 0
    g.close()
    o.close()


def test_unknown_and_max_distance_bit_exact():
    eps = float(V)
    obs = lambda c: (c[..., 2] < 0.8) | (c[..., 2] > 1.2)  # noqa: E731
    keys, D, W, _ = tsdf_region((0, 0, 0), (2, 2, 4), lambda c: c[..., 2] - 0.43, observed=obs)
    g, o = _pair(V, eps, 5)
    _, st = _step(g, o, keys, D, W, None, eps, 5)
    assert (st == 0).any() and ((st & ESDF_OBS) != 0).any() and ((st & ESDF_PAR) == 0).any()
    g.close()
    o.close()


@pytest.fixture(scope="module")
def room_tsdf():
    """The oracle's TSDF of room frames 0-19 and 0-39 (FP64 rounded to FP32)."""
    w = synth.config_room(n_frames=300)
    m = oracle.OracleMap(w.voxel_size)
    out = []
    for k, f in enumerate(w.frames[:40]):
        m.integrate(f.sensor, f.T, f.depth)
        if k in (19, 39):
            keys, D, W = m.export()
            out.append((keys, D.astype(np.float32), W.astype(np.float32)))
    m.close()
    return w, out


def test_room_incremental_bit_exact(room_tsdf):
    """ESDF of the room after 20 frames, then after 20 more (new and changed
    blocks imported), against the oracle; site threshold 1 voxel, 48-voxel
    range."""
    w, ((k1, D1, W1), (k2, D2, W2)) = room_tsdf
    v = np.float32(w.voxel_size)
    eps, md = float(v), 48
    g, o = _pair(v, eps, md, max_blocks=1 << 16)
    _step(g, o, k1, D1, W1, None, eps, md)
    # second state: blocks that are new or whose values changed
    idx = {tuple(k): i for i, k in enumerate(k1)}
    changed = np.ones(len(k2), bool)
    for j, k in enumerate(k2):
        i = idx.get(tuple(k))
        if i is not None:
            changed[j] = not (np.array_equal(D1[i], D2[j]) and np.array_equal(W1[i], W2[j]))
    assert 0 < changed.sum() < len(k2)
    _, st = _step(g, o, k2, D2, W2, changed, eps, md)
    stats = g.esdf_stats()
    assert stats["iterations"] >= 4 and stats["cleared"] > 0
    assert ((st & ESDF_PAR) != 0).sum() > 100000
    g.close()
    o.close()


def test_query_matches_export():
    eps = float(V)
    keys, D, W, _ = tsdf_region((0, 0, 0), (3, 3, 3),
                                lambda c: np.linalg.norm(c - np.array([0.6, 0.6, 0.6]), axis=-1) - 0.4,
                                observed=lambda c: c[..., 0] < 1.0)
    g = gt.TsdfMap(float(V))
    g.import_blocks(keys, D, W)
    g.esdf_update(eps, 1e-4, 20)
    k, st = g.esdf_export()
    off = esdf_offsets(st)
    d = np.sqrt((off.astype(np.float64) ** 2).sum(-1)).astype(np.float32)
    d = np.where((st & ESDF_PAR) != 0, d, np.float32(20))
    d = np.where((st & ESDF_INSIDE) != 0, -d, d) * np.float32(V)
    d = np.where((st & ESDF_OBS) != 0, d, np.nan).astype(np.float32)
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    centres = ((k[:, None, :] * 8 + loc[None]) + 0.5) * float(V)
    pts = torch.from_numpy(centres.reshape(-1, 3).astype(np.float32)).cuda()
    out = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    g.esdf_query(pts, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), d.reshape(-1))
    far = torch.tensor([[50.0, 50.0, 50.0]], dtype=torch.float32, device="cuda")
    g.esdf_query(far, out[:1])
    assert torch.isnan(out[:1]).all()
    g.close()


@pytest.mark.parametrize("storage", [gt.STORAGE_FP32, gt.STORAGE_FP16, gt.STORAGE_FIXED16])
def test_room_gpu_integrated_properties(storage):
    """GPU integration then GPU ESDF on 30 room frames: every parent is a
    site, site flags follow |D| <= eps on the GPU's own TSDF, no distance is
    below the Euclidean distance to the nearest site (sampled voxels)."""
    from scipy.spatial import cKDTree
    w = synth.config_room(n_frames=300)
    v = float(np.float32(w.voxel_size))
    g = gt.TsdfMap(w.voxel_size, storage=storage)
    for f in w.frames[:30]:
        g.integrate(f.sensor, f.T, torch.from_numpy(np.ascontiguousarray(f.depth)).cuda())
    g.esdf_update(v, 1e-4, 40)
    keys, D, W = g.export()
    k2, st = g.esdf_export()
    np.testing.assert_array_equal(keys, k2)
    site = (st & ESDF_SITE) != 0
    np.testing.assert_array_equal(site, (W >= np.float32(1e-4)) & (np.abs(D) <= np.float32(v)))
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    gidx = keys[:, None, :] * 8 + loc[None]
    par = (st & ESDF_PAR) != 0
    parent = gidx + esdf_offsets(st)
    site_pts = gidx[site]
    tree = cKDTree(site_pts)
    # every parent is a site
    d_par, _ = tree.query(parent[par][::7], k=1)
    assert np.all(d_par == 0)
    # never below the exact distance
    rng = np.random.default_rng(0)
    sel = rng.choice(np.flatnonzero(par.reshape(-1)), 20000, replace=False)
    exact, _ = tree.query(gidx.reshape(-1, 3)[sel], k=1)
    got = np.sqrt((esdf_offsets(st).reshape(-1, 3)[sel].astype(np.float64) ** 2).sum(-1))
    assert np.all(got >= exact - 1e-9)
    # (propagation runs through observed voxels of allocated blocks only, so
    # a voxel may reach its nearest site only by a detour: no equality bound)
    g.close()


def test_esdf_argument_errors():
    col = gt.TsdfMap(float(V), layer=gt.LAYER_COLOR)  # colour maps have no ESDF
    with pytest.raises(gt.TsdfError):
        col.esdf_update()
    col.close()
    g = gt.TsdfMap(float(V))
    with pytest.raises(gt.TsdfError):  # nothing to export before the first update
        g.esdf_export()
    g.esdf_update(float(V), 1e-4, 30)
    with pytest.raises(gt.TsdfError):  # parameters are fixed by the first update
        g.esdf_update(float(V), 1e-4, 31)
    with pytest.raises(gt.TsdfError):
        g.esdf_update(float(V), 1e-4, 256)
    keys = np.array([[0, 0, 0], [0, 0, 0]], np.int32)
    with pytest.raises(gt.TsdfError):  # duplicate keys
        g.import_blocks(keys, np.zeros((2, 512), np.float32), np.zeros((2, 512), np.float32))
    g.close()
