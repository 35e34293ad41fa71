"""GPU parity of the ESDF of occupancy layers (Sec. IV-C: an occupancy voxel
is a site if it is adjacent to free voxels) against the oracle, through the
C ABI.

Log-odds l > 0 is occupied (inside), l < 0 free, l = 0 unknown; a site is an
occupied voxel with a free face neighbour, possibly in the next block.  Both
sides start from the same FP32 log-odds: layers written from closed-form
regions and imported with map_import, or integrated by the GPU's occupancy
functor (room frames, decay steps) and exported.  The ESDF arithmetic is
integer, so voxel states and the iteration, sweep, exchange and clearing
counts must match bit for bit, including incremental updates where only a
face neighbour of a block changed.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from tests.esdf_inputs import V, occupancy_region

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2311_00626_gb300 as gt  # noqa: E402
from oracle import ESDF_PAR, ESDF_SITE  # noqa: E402


def _pair(v, max_dist, max_blocks=1 << 14):
    g = gt.TsdfMap(float(v), max_blocks=max_blocks, layer=gt.LAYER_OCCUPANCY)
    o = oracle.EsdfOracle(float(v), 0.0, 0.0, max_dist, occupancy=True)
    return g, o


def _compare(g, o):
    gk, gs = g.esdf_export()
    ok, os_ = o.export()
    np.testing.assert_array_equal(gk, ok)
    bad = np.count_nonzero(gs != os_)
    assert bad == 0, f"{bad} ESDF voxel states differ"
    gc, oc = g.esdf_stats(), o.counters()
    assert gc == oc, (gc, oc)
    return gk, gs


def _step(g, o, keys, L, changed, max_dist):
    """Import the changed blocks into the GPU map, update both layers,
    compare states and counters."""
    ch = np.ones(len(keys), bool) if changed is None else changed
    g.import_blocks(keys[ch], L[ch])
    g.esdf_update(float(V), 1e-4, max_dist)
    o.update(keys, L, np.zeros_like(L), ch)
    return _compare(g, o)


def test_closed_form_layers_bit_exact():
    """Half-space (sites on a block face), a box in free space, and an
    unknown slab between occupied and free space (no sites at all)."""
    cases = [  # occupied, known, block range, whether sites exist
        (lambda c: c[..., 2] < 0.4, None, (0, 0, 0), (3, 3, 4), True),
        (lambda c: np.all((c >= 10 * float(V)) & (c < 18 * float(V)), axis=-1), None, (0, 0, 0), (4, 4, 4), True),
        (lambda c: c[..., 2] < 0.4, lambda c: (c[..., 2] < 0.4) | (c[..., 2] >= 0.6), (0, 0, 0), (2, 2, 4), False),
        (lambda c: np.linalg.norm(c - np.array([-0.3, 0.2, -0.6]), axis=-1) < 0.4, None, (-3, -2, -4), (1, 2, 0),
         True),
    ]
    for occ, known, lo, hi, has_sites in cases:
        keys, L, _ = occupancy_region(lo, hi, occ, known)
        g, o = _pair(V, 60)
        _, st = _step(g, o, keys, L, None, 60)
        assert np.any(st & ESDF_SITE) == has_sites
        g.close()
        o.close()


def test_incremental_neighbour_block_bit_exact():
    """Occupied below z = 0.4 m, then below 0.5 m: only the blocks above the
    face are imported again, and the sites of the unchanged blocks below it
    vanish (their +z neighbours turned occupied)."""
    keys, L1, g_idx = occupancy_region((0, 0, 0), (3, 2, 4), lambda c: c[..., 2] < 0.4)
    _, L2, _ = occupancy_region((0, 0, 0), (3, 2, 4), lambda c: c[..., 2] < 0.5)
    changed = np.any(L1 != L2, axis=1)
    assert not np.any(changed[keys[:, 2] == 0])
    g, o = _pair(V, 40)
    _step(g, o, keys, L1, None, 40)
    k, st = _step(g, o, keys, L2, changed, 40)
    assert g.esdf_stats()["cleared"] > 0
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    np.testing.assert_array_equal((st & ESDF_SITE) != 0, g_idx[order][..., 2] == 9)
    g.close()
    o.close()


def _export_changed(prev, keys, L):
    """Blocks new since `prev` (keys -> values) or with changed values."""
    if prev is None:
        return np.ones(len(keys), bool)
    out = np.zeros(len(keys), bool)
    for i, k in enumerate(map(tuple, keys.tolist())):
        p = prev.get(k)
        out[i] = p is None or not np.array_equal(p, L[i])
    return out


def test_room_occupancy_integrated_and_decayed_bit_exact():
    """Occupancy layer integrated on the GPU from 20 room frames, ESDF on
    both sides from its exported log-odds; then a decay step and 5 more
    frames, and an incremental update on both sides (the oracle told which
    blocks changed value; the GPU marks what integration and decay
    flagged)."""
    w = synth.config_room(n_frames=300)
    v = float(np.float32(w.voxel_size))
    g = gt.TsdfMap(w.voxel_size, w.truncation_voxels, w.max_weight, layer=gt.LAYER_OCCUPANCY)
    o = oracle.EsdfOracle(v, 0.0, 0.0, 40, occupancy=True)
    prev = None
    for frames, decay in ((w.frames[:20], False), (w.frames[20:25], True)):
        if decay:
            g.decay(0.3, 0.1)
        for f in frames:
            g.integrate(f.sensor, f.T, torch.from_numpy(np.ascontiguousarray(f.depth)).cuda())
        torch.cuda.synchronize()
        keys, L, _ = g.export()
        ch = _export_changed(prev, keys, L)
        g.esdf_update(v, 1e-4, 40)
        o.update(keys, L, np.zeros_like(L), ch)
        _, st = _compare(g, o)
        prev = {k: L[i].copy() for i, k in enumerate(map(tuple, keys.tolist()))}
        assert np.any(st & ESDF_SITE) and np.any(st & ESDF_PAR)
    g.close()
    o.close()


def test_decay_to_unknown_clears_sites():
    """Decay that takes every log-odds to 0 leaves every voxel unknown: no
    sites, no parents, on both sides."""
    keys, L, _ = occupancy_region((0, 0, 0), (2, 2, 2), lambda c: c[..., 2] < 0.4)
    g, o = _pair(V, 20)
    _step(g, o, keys, L, None, 20)
    g.decay(10.0, 10.0)
    torch.cuda.synchronize()
    k2, L2, _ = g.export()
    assert np.all(L2 == 0)
    g.esdf_update(float(V), 1e-4, 20)
    o.update(k2, L2, np.zeros_like(L2), np.ones(len(k2), bool))
    _, st = _compare(g, o)
    assert np.all(st == 0)
    g.close()
    o.close()
