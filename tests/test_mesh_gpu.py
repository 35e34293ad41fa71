"""GPU parity of marching-cubes meshing against the oracle, through the C ABI.

Both sides mesh the same FP32 TSDF (imported into the GPU map).  Which
cubes are meshed, their case and the triangles' vertex edges are integer
decisions on the same values, so the triangle sets (cube and vertex keys)
must be equal; vertex positions are FP32 on the GPU and FP64 in the oracle
and agree within a few units in the last place of the coordinates.
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


def _canon(cube, keys, pos):
    """Sort triangles by (cube, vertex keys) so both sides line up."""
    rec = np.concatenate([cube.reshape(len(cube), -1), keys.reshape(len(keys), -1)], 1).astype(np.int64)
    order = np.lexsort(rec.T[::-1])
    return rec[order], pos[order]


def _compare(g_out, o_out, v):
    gp, gk, gc = (x.cpu().numpy() for x in g_out)
    oc, ok, op = o_out
    assert len(gk) == len(ok), (len(gk), len(ok))
    grec, gpos = _canon(gc, gk, gp.astype(np.float64))
    orec, opos = _canon(oc, ok, op)
    np.testing.assert_array_equal(grec, orec)
    tol = 4 * np.spacing(np.abs(opos).astype(np.float32)).astype(np.float64) + float(v) * 2.0 ** -20
    assert np.all(np.abs(gpos - opos) <= tol), np.abs(gpos - opos).max()
    return len(gk)


def _map(v, storage=gt.STORAGE_FP32, max_blocks=1 << 14):
    return gt.TsdfMap(float(v), storage=storage, max_blocks=max_blocks)


@pytest.mark.parametrize("name", ["plane", "sphere", "random"])
def test_shapes_bit_exact(name):
    if name == "plane":
        keys, D, W, _ = tsdf_region((0, 0, 0), (3, 3, 2), lambda c: c[..., 2] - 0.43)
    elif name == "sphere":
        keys, D, W, _ = tsdf_region((-2, 0, -1), (2, 3, 2),
                                    lambda c: np.linalg.norm(c - np.array([-0.1, 0.6, 0.05]), axis=-1) - 0.45)
    else:
        rng = np.random.default_rng(4)
        keys, D, W, g = tsdf_region((0, 0, 0), (2, 2, 2), lambda c: np.zeros(c.shape[:-1]))
        D = rng.normal(size=(16, 16, 16)).astype(np.float32)[g[..., 0], g[..., 1], g[..., 2]]
        W[rng.uniform(size=W.shape) < 0.05] = 0.0  # some unobserved voxels
    m = _map(V)
    m.import_blocks(keys, D, W)
    n = _compare(m.mesh(), oracle.mesh_extract(keys, D, W, float(V)), V)
    assert n > 100
    m.close()


def test_changed_only_incremental():
    """A sphere, then its part beyond x = 0.85 m shrunk by 3 cm: with
    changed_only the GPU meshes the re-imported blocks and the blocks whose
    cubes reach into them."""
    f1 = lambda c: np.linalg.norm(c - np.array([0.6, 0.6, 0.6]), axis=-1) - 0.35  # noqa: E731
    f2 = lambda c: np.where(c[..., 0] > 0.85, f1(c) + 0.03, f1(c))  # noqa: E731
    keys, D1, W, _ = tsdf_region((0, 0, 0), (3, 3, 3), f1)
    _, D2, _, _ = tsdf_region((0, 0, 0), (3, 3, 3), f2)
    m = _map(V)
    m.import_blocks(keys, D1, W)
    _compare(m.mesh(changed_only=True), oracle.mesh_extract(keys, D1, W, float(V)), V)
    # nothing changed: nothing to mesh
    assert len(m.mesh(changed_only=True)[0]) == 0
    changed = np.any(D1 != D2, axis=1)
    assert 0 < changed.sum() < len(keys)
    m.import_blocks(keys[changed], D2[changed], W[changed])
    ch = {tuple(k) for k in keys[changed].tolist()}
    sel = np.array([any((x + dx, y + dy, z + dz) in ch for dx in (0, 1) for dy in (0, 1) for dz in (0, 1))
                    for x, y, z in keys.tolist()])
    _compare(m.mesh(changed_only=True), oracle.mesh_extract(keys, D2, W, float(V), blocks=sel), V)
    m.close()


def test_fp16_storage():
    """FP16 map: both sides mesh the values as stored (D / tau and W rounded
    to half precision, decoded as half * tau in FP32)."""
    keys, D, W, _ = tsdf_region((0, 0, 0), (3, 3, 3),
                                lambda c: np.linalg.norm(c - np.array([0.6, 0.61, 0.59]), axis=-1) - 0.4)
    tau = np.float32(4 * float(V))
    inv = np.float32(1.0) / tau
    D16 = ((D.astype(np.float32) * inv).astype(np.float16).astype(np.float32) * tau).astype(np.float32)
    W16 = W.astype(np.float16).astype(np.float32)
    m = _map(V, storage=gt.STORAGE_FP16)
    m.import_blocks(keys, D, W)
    _compare(m.mesh(), oracle.mesh_extract(keys, D16, W16, float(V)), V)
    m.close()


def test_fixed16_storage():
    """16-bit fixed-point map: both sides mesh the values as stored (D / tau
    rounded to 1 / 32767, W to half precision, decoded in FP32)."""
    keys, D, W, _ = tsdf_region((0, 0, 0), (3, 3, 3),
                                lambda c: np.linalg.norm(c - np.array([0.61, 0.6, 0.58]), axis=-1) - 0.4)
    tau = np.float32(4.0 * float(np.float32(V)))
    scale = np.float32(32767.0 / float(tau))
    unit = np.float32(float(tau) / 32767.0)
    q = np.rint(np.clip((D.astype(np.float32) * scale).astype(np.float32), -32767, 32767))
    Dq = (q.astype(np.float32) * unit).astype(np.float32)
    W16 = W.astype(np.float16).astype(np.float32)
    m = _map(V, storage=gt.STORAGE_FIXED16)
    m.import_blocks(keys, D, W)
    k2, D2, W2 = m.export()
    np.testing.assert_array_equal(W2, W16)
    np.testing.assert_array_equal(D2, Dq)
    _compare(m.mesh(), oracle.mesh_extract(keys, Dq, W16, float(V)), V)
    m.close()


def test_room_from_oracle_tsdf():
    """The oracle's TSDF of 20 room frames (FP64 rounded to FP32), meshed
    on both sides."""
    w = synth.config_room(n_frames=300)
    om = oracle.OracleMap(w.voxel_size)
    for f in w.frames[:20]:
        om.integrate(f.sensor, f.T, f.depth)
    keys, D, W = om.export()
    om.close()
    D, W = D.astype(np.float32), W.astype(np.float32)
    v = np.float32(w.voxel_size)
    m = _map(v, max_blocks=1 << 16)
    m.import_blocks(keys, D, W)
    n = _compare(m.mesh(), oracle.mesh_extract(keys, D, W, float(v)), v)
    assert n > 100000
    m.close()


def test_capacity_and_errors():
    keys, D, W, _ = tsdf_region((0, 0, 0), (2, 2, 2), lambda c: c[..., 2] - 0.43)
    m = _map(V)
    m.import_blocks(keys, D, W)
    full = len(m.mesh()[0])
    with pytest.raises(gt.TsdfError):
        m.mesh(cap=10, changed_only=True)  # capacity: reported, not retried
    occ = gt.TsdfMap(float(V), layer=gt.LAYER_OCCUPANCY)
    with pytest.raises(gt.TsdfError):
        occ.mesh()
    occ.close()
    assert full > 10
    m.close()


def test_gpu_integrated_room_mesh_properties():
    """After GPU integration of 20 room frames: every vertex lies on its
    cube edge, between the edge's two voxel centres."""
    w = synth.config_room(n_frames=300)
    v = float(np.float32(w.voxel_size))
    m = gt.TsdfMap(w.voxel_size)
    for f in w.frames[:20]:
        m.integrate(f.sensor, f.T, torch.from_numpy(np.ascontiguousarray(f.depth)).cuda())
    pos, keys, _ = (x.cpu().numpy() for x in m.mesh())
    assert len(pos) > 100000
    lo = (keys[..., :3] + 0.5) * v
    ax = keys[..., 3]
    for a in range(3):
        along = ax == a
        assert np.all(np.abs(pos[..., a][~along] - lo[..., a][~along]) <= 4 * np.spacing(np.float32(20.0)))
        d = pos[..., a][along] - lo[..., a][along]
        assert np.all(d >= -1e-6) and np.all(d <= v + 1e-6)
    m.close()
